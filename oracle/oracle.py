"""ctypes marshalling for the FP64 oracle (``pvg_oracle.c``).

Test infrastructure only: see the package docstring.  Inputs are the scene
and camera dicts of ``paper_2311_18561_gb300.synth`` (any float type); they
are converted to float64 here and every output is float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pvg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libpvg_oracle.so")

# Options (3DGS conventions the paper inherits): EWA dilation h [px^2],
# alpha cap, alpha gate, transmittance stop, frustum clamp factor.
DEFAULT_OPTS = dict(h=0.3, alpha_cap=0.99, alpha_min=1.0 / 255.0, t_stop=1e-4, fov_clamp=1.3)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        lib.pvgo_time_eval.argtypes = [C.c_int64] + [P] * 6 + [C.c_double, C.c_double, P, P]
        lib.pvgo_sh_basis.argtypes = [C.c_int, C.c_int64, P, P, P]
        lib.pvgo_preprocess.argtypes = [C.c_int64, C.c_int] + [P] * 11 + [P] * 9
        sky = [P, C.c_int, P]
        feat = [C.c_int, C.c_int, P]
        lib.pvgo_render.argtypes = ([C.c_int64, C.c_int] + [P] * 11 + [C.c_int, C.c_int64, P] + sky + feat
                                    + [P] * 7)
        lib.pvgo_render_bwd.argtypes = ([C.c_int64, C.c_int] + [P] * 11 + [C.c_int, C.c_int64, P] + sky
                                        + feat + [P] + [P] * 3 + [P] * 12)
        lib.pvgo_num_threads.argtypes = []
        for f in (lib.pvgo_time_eval, lib.pvgo_sh_basis, lib.pvgo_preprocess, lib.pvgo_render,
                  lib.pvgo_render_bwd, lib.pvgo_num_threads):
            f.restype = C.c_int
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(load().pvgo_num_threads())


def cam_array(cam) -> np.ndarray:
    """viewmat[12], fx, fy, cx, cy, width, height, t, z_near, bg[3], dt."""
    vm = np.asarray(cam["viewmat"], np.float64).reshape(12)
    rest = [cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"], cam["height"],
            cam["t"], cam["z_near"]]
    return np.concatenate([vm, np.asarray(rest, np.float64), np.asarray(cam["bg"], np.float64).reshape(3),
                           np.asarray([float(cam.get("dt", 0.0))])])


def opt_array(opts=None) -> np.ndarray:
    o = dict(DEFAULT_OPTS)
    if opts:
        o.update(opts)
    return np.asarray([o["h"], o["alpha_cap"], o["alpha_min"], o["t_stop"], o["fov_clamp"]], np.float64)


def _scene_args(scene):
    k = scene["sh"].shape[1]
    deg = int(round(np.sqrt(k))) - 1
    arrs = [_d(scene[name]) for name in ("mu", "vel", "tau", "beta", "period", "scale", "quat",
                                         "opacity", "sh")]
    return int(scene["mu"].shape[0]), deg, arrs


def time_eval(scene, t, dt=0.0):
    """Eq. 6 and Eq. 7: (mu~(t) [N,3], o~(t) [N]); with dt != 0 the
    flow-translated state of Sec. 3.4 (queried at t - dt, moved by
    v_bar dt)."""
    n = int(np.asarray(scene["mu"]).shape[0])
    arrs = [_d(scene[k]) for k in ("mu", "vel", "tau", "beta", "period", "opacity")]
    mut = np.zeros((n, 3))
    ot = np.zeros(n)
    load().pvgo_time_eval(n, *[_p(a) for a in arrs], float(t), float(dt), _p(mut), _p(ot))
    return mut, ot


def sh_basis(degree, dirs):
    """Real SH basis values [n, K] and polynomial gradients [n, K, 3]."""
    dirs = _d(dirs).reshape(-1, 3)
    k = (degree + 1) ** 2
    Y = np.zeros((dirs.shape[0], k))
    dY = np.zeros((dirs.shape[0], k, 3))
    rc = load().pvgo_sh_basis(int(degree), dirs.shape[0], _p(dirs), _p(Y), _p(dY))
    if rc != 0:
        raise ValueError("bad SH degree")
    return Y, dY


def preprocess(scene, cam, opts=None):
    """Steps 1-4 per Gaussian: dict of valid, mut, ot, pcam, uv, cov2, conic,
    rgb, box (rx, ry)."""
    n, deg, arrs = _scene_args(scene)
    out = dict(valid=np.zeros(n, np.int32), mut=np.zeros((n, 3)), ot=np.zeros(n),
               pcam=np.zeros((n, 3)), uv=np.zeros((n, 2)), cov2=np.zeros((n, 3)),
               conic=np.zeros((n, 3)), rgb=np.zeros((n, 3)), box=np.zeros((n, 2)))
    ca, oa = cam_array(cam), opt_array(opts)
    rc = load().pvgo_preprocess(n, deg, *[_p(a) for a in arrs], _p(ca), _p(oa),
                                *[_p(out[k]) for k in ("valid", "mut", "ot", "pcam", "uv", "cov2",
                                                       "conic", "rgb", "box")])
    if rc != 0:
        raise ValueError("oracle preprocess rejected its inputs")
    return out


def _sky_args(sky, jitter):
    """sky: None or [6, R, R, 3] cube map; jitter: None or [2, H, W] pixel
    offsets of the sky rays."""
    if sky is None:
        return None, 0, None, None
    sk = _d(sky)
    jt = None if jitter is None else _d(jitter)
    return sk, int(sk.shape[1]), jt, (_p(sk), int(sk.shape[1]), _p(jt))


# extra channels of step 8 (bit flags): v_bar (3), rho clamped to [0, 2] (1),
# semantic vector (n_sem)
FEAT_VBAR, FEAT_RHO, FEAT_SEM = 1, 2, 4


def feat_count(mask, n_sem=0):
    return (3 if mask & FEAT_VBAR else 0) + (1 if mask & FEAT_RHO else 0) + (n_sem if mask & FEAT_SEM else 0)


def _feat_args(features, sem):
    """features: channel mask; sem: [N, S] semantic vectors (FEAT_SEM)."""
    mask = int(features or 0)
    if mask & FEAT_SEM:
        if sem is None:
            raise ValueError("FEAT_SEM needs the semantic vectors")
        sm = _d(sem)
        return mask, int(sm.shape[1]), sm
    return mask, 0, None


def render(scene, cam, opts=None, mode="brute", pixels=None, sky=None, sky_jitter=None, features=0, sem=None):
    """Steps 5/6 (and 8).  mode 'brute' or 'culled'.  pixels: None for the
    full image (outputs shaped [H, W, ...]) or an int array [P, 2] of
    (px, py) (outputs shaped [P, ...]).  sky: optional cube map (see
    _sky_args).  features: mask of FEAT_* channels (sem: [N, S] for
    FEAT_SEM), returned as 'feat' [..., F].
    Returns dict rgb, depth, alpha, T, nblend, flag (, feat)."""
    n, deg, arrs = _scene_args(scene)
    fmask, nsem, sm = _feat_args(features, sem)
    F = feat_count(fmask, nsem)
    sk, res, jt, skp = _sky_args(sky, sky_jitter)
    if skp is None:
        skp = (None, 0, None)
    W, H = int(cam["width"]), int(cam["height"])
    if pixels is None:
        P = W * H
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        P = pix.shape[0]
    out = dict(rgb=np.zeros((P, 3)), depth=np.zeros(P), alpha=np.zeros(P), T=np.zeros(P),
               nblend=np.zeros(P, np.int32), flag=np.zeros(P, np.int32))
    if F:
        out["feat"] = np.zeros((P, F))
    ca, oa = cam_array(cam), opt_array(opts)
    m = {"brute": 0, "culled": 1}[mode]
    rc = load().pvgo_render(n, deg, *[_p(a) for a in arrs], _p(ca), _p(oa), m, P, _p(pix), *skp,
                            fmask, nsem, _p(sm),
                            *[_p(out[k]) for k in ("rgb", "depth", "alpha", "T", "nblend", "flag")],
                            _p(out.get("feat")))
    if rc != 0:
        raise ValueError("oracle render rejected its inputs")
    if pixels is None:
        out = {k: v.reshape((H, W) + v.shape[1:]) for k, v in out.items()}
    return out


GRAD_NAMES = ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh")


def render_bwd(scene, cam, dL_rgb, dL_depth, dL_alpha, opts=None, return_g2d=False, mode="brute",
               pixels=None, sky=None, sky_jitter=None, features=0, sem=None, dL_feat=None):
    """Gradients of sum(dL_rgb*rgb) + sum(dL_depth*depth) + sum(dL_alpha*alpha)
    (+ sum(dL_feat*feat) for the channels in ``features``) w.r.t. every
    parameter, as a dict keyed like the scene (plus 'sem' for FEAT_SEM).
    Full image (dL_rgb [H,W,3], others [H,W], dL_feat [H,W,F]) or, with
    ``pixels`` [P,2], only those pixels (dL_rgb [P,3], others [P],
    dL_feat [P,F]).  mode 'brute' or 'culled'."""
    n, deg, arrs = _scene_args(scene)
    fmask, nsem, sm = _feat_args(features, sem)
    F = feat_count(fmask, nsem)
    gf = _d(dL_feat) if F else None
    dsem = np.zeros((n, nsem)) if fmask & FEAT_SEM else None
    k = (deg + 1) ** 2
    g = dict(mu=np.zeros((n, 3)), vel=np.zeros((n, 3)), tau=np.zeros(n), beta=np.zeros(n),
             period=np.zeros(n), scale=np.zeros((n, 3)), quat=np.zeros((n, 4)), opacity=np.zeros(n),
             sh=np.zeros((n, k, 3)))
    g2d = np.zeros((n, 10))
    ca, oa = cam_array(cam), opt_array(opts)
    gr, gd, ga = _d(dL_rgb), _d(dL_depth), _d(dL_alpha)
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
    npix = 0 if pix is None else pix.shape[0]
    m = {"brute": 0, "culled": 1}[mode]
    sk, res, jt, skp = _sky_args(sky, sky_jitter)
    dsky = None
    if skp is None:
        skp = (None, 0, None)
    else:
        dsky = np.zeros_like(sk)
        g["sky"] = dsky
    rc = load().pvgo_render_bwd(n, deg, *[_p(a) for a in arrs], _p(ca), _p(oa), m, npix, _p(pix), *skp,
                                fmask, nsem, _p(sm), _p(gf), _p(gr), _p(gd), _p(ga),
                                *[_p(g[name]) for name in GRAD_NAMES], _p(g2d), _p(dsky), _p(dsem))
    if rc != 0:
        raise ValueError("oracle backward rejected its inputs")
    if dsem is not None:
        g["sem"] = dsem
    if return_g2d:
        return g, g2d
    return g
