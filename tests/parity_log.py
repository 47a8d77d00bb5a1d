"""Record of every GPU-vs-oracle image comparison of a test session (test,
pixels compared, pixels the oracle flagged, largest errors), printed in
pytest's terminal summary so that a run's log shows the real flagged
fractions.  Plain Python: importable without torch."""
import os

RECORDS = []


def record(kind, compared, flagged, **errors):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    RECORDS.append(dict(test=test, kind=kind, compared=int(compared), flagged=int(flagged),
                        errors={k: float(v) for k, v in errors.items()}))


def summary_lines():
    if not RECORDS:
        return []
    total = sum(r["compared"] for r in RECORDS)
    flagged = sum(r["flagged"] for r in RECORDS)
    out = ["%d image comparisons with the oracle: %d of %d pixels flagged (%.4f %%)"
           % (len(RECORDS), flagged, total, 100.0 * flagged / max(1, total))]
    for r in RECORDS:
        errs = " ".join("%s=%.2e" % kv for kv in sorted(r["errors"].items()))
        out.append("  %-5s %7d px  flagged %5d (%.4f %%)  %s  %s"
                   % (r["kind"], r["compared"], r["flagged"], 100.0 * r["flagged"] / max(1, r["compared"]),
                      errs, r["test"]))
    return out
