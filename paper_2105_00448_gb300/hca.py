"""Thin ctypes binding of libhca.so (include/hca.h).

Only argument marshalling lives here: every step of the hot path runs in the
library's CUDA kernels.  Host buffers are numpy arrays; device buffers are
torch CUDA tensors (PyTorch supplies device memory and streams only).  There
is no CPU fallback: if libhca.so cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import os
import struct
from typing import Dict, Optional, Sequence

import numpy as np

from . import _build

# status codes (hca.h)
HCA_OK = 0
HCA_ERR_ARG = -1
HCA_ERR_CUDA = -2
HCA_ERR_OOM = -3
HCA_ERR_NONFINITE = -4
HCA_ERR_NOCONV = -5
HCA_ERR_TIMEOUT = -6
HCA_ERR_UNIMPLEMENTED = -7
HCA_ERR_STATE = -8
HCA_ERR_IO = -9

HCA_FP64 = 0
HCA_FP32 = 1
HCA_WS_PREV = 0
HCA_WS_LEARNED = 1
HCA_WS_LEARNED_ALWAYS = 2
HCA_PC_JACOBI = 0
HCA_PC_MG = 1

EMPTY, PROLIF, QUIESC, DEAD, VESSEL, STROMA = range(6)

FIELD_O2 = 1 << 0
FIELD_DRUG0 = 1 << 1
FIELD_DRUG1 = 1 << 2
FIELD_DRUG2 = 1 << 3
FIELD_PHI = 1 << 4
FIELD_P53 = 1 << 5
FIELD_VEGFC = 1 << 6
FIELD_PERF = 1 << 7
FIELD_VEGF = 1 << 8
# low-order words of the FP32 defect-correction fields (read only)
FIELD_O2_LO = 1 << 9
FIELD_DRUG0_LO = 1 << 10
FIELD_DRUG1_LO = 1 << 11
FIELD_DRUG2_LO = 1 << 12
FIELD_VEGF_LO = 1 << 13
FIELD_DRUG = (FIELD_DRUG0, FIELD_DRUG1, FIELD_DRUG2)

STAGE_O2 = 1 << 0
STAGE_DRUGS = 1 << 1
STAGE_ODE = 1 << 2
STAGE_CA = 1 << 3
STAGE_ADVANCE = 1 << 4
STAGE_ALL = 0x1F

_d3 = ctypes.c_double * 3
_i3 = ctypes.c_int32 * 3


class hca_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("n_drugs", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("rtol_o2", ctypes.c_double), ("rtol_drug", ctypes.c_double),
        ("maxit", ctypes.c_int32), ("ode_substeps", ctypes.c_int32),
        ("picard_tol", ctypes.c_double), ("picard_maxit", ctypes.c_int32),
        ("dose_interval", ctypes.c_int32),
        ("D_K", ctypes.c_double), ("phi_K", ctypes.c_double), ("K1", ctypes.c_double),
        ("K0", ctypes.c_double), ("r_K", ctypes.c_double),
        ("D_G", _d3), ("psi_G", _d3), ("kappa_G", _d3), ("uptake_G", _d3),
        ("dose_peak", _d3), ("plasma_decay", _d3), ("kill_b", _i3),
        ("T_cycle", ctypes.c_double), ("K_phi", ctypes.c_double),
        ("k1", ctypes.c_double), ("k1p", ctypes.c_double), ("K_p53", ctypes.c_double),
        ("k2", ctypes.c_double), ("k2p", ctypes.c_double), ("k2pp", ctypes.c_double),
        ("J5", ctypes.c_double), ("K_V", ctypes.c_double),
        ("rtol_inner", ctypes.c_double), ("max_outer", ctypes.c_int32),
        ("warm_start", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
        ("threads_per_block", ctypes.c_int32), ("o2_nonlinear", ctypes.c_int32),
        ("drug_scheme", ctypes.c_int32), ("drug_substeps", ctypes.c_int32),
        ("o2_scheme", ctypes.c_int32), ("o2_substeps", ctypes.c_int32), ("ca_mode", ctypes.c_int32),
        ("vegf", ctypes.c_int32), ("vessel_interval", ctypes.c_int32), ("pk_model", _i3), ("pad3", ctypes.c_int32),
        ("D_V", ctypes.c_double), ("psi_V", ctypes.c_double), ("a_V", ctypes.c_double),
        ("V_low", ctypes.c_double), ("V_high", ctypes.c_double),
        ("p_death", ctypes.c_double), ("beta_birth", ctypes.c_double), ("V_sprout", ctypes.c_double),
        ("mm_vmax", ctypes.c_double), ("mm_km", ctypes.c_double), ("epi_w", _d3),
        ("epi_q2", ctypes.c_double), ("epi_q3", ctypes.c_double), ("epi_cl2", ctypes.c_double),
        ("stream", ctypes.c_void_p),
    ]


class hca_stats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("picard_iterations", ctypes.c_int32),
        ("o2_iterations", ctypes.c_int32),
        ("o2_sweeps", ctypes.c_int32),
        ("drug_iterations", _i3),
        ("o2_rel_residual", ctypes.c_double),
        ("drug_rel_residual", _d3),
        ("not_converged", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("committed", ctypes.c_int64), ("kills", ctypes.c_int64),
        ("divisions", ctypes.c_int64), ("blocked", ctypes.c_int64),
        ("counts", ctypes.c_int64 * 6),
        ("ws_used", ctypes.c_int32),
        ("pad1", ctypes.c_int32),
        ("ws_r0_prev", ctypes.c_double),
        ("ws_r0_learned", ctypes.c_double),
        ("vegf_iterations", ctypes.c_int32), ("pad2", ctypes.c_int32),
        ("vegf_rel_residual", ctypes.c_double),
        ("vessel_births", ctypes.c_int64), ("vessel_deaths", ctypes.c_int64),
    ]

    def as_dict(self) -> Dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


NKCLASS = 13
KCLASS_NAMES = ("setup", "pass_a", "pass_b", "residual", "ode", "ca_compact", "ca_colour", "other", "mg",
                "mg_restrict0", "mg_post0", "mg_pre0", "mg_last0")


class hca_train_cfg(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("n_samples", ctypes.c_int32),
                ("state", ctypes.POINTER(ctypes.c_void_p)), ("perf", ctypes.POINTER(ctypes.c_void_p)),
                ("K_prev", ctypes.POINTER(ctypes.c_void_p)), ("K_new", ctypes.POINTER(ctypes.c_void_p)),
                ("iters", ctypes.c_int32), ("lr", ctypes.c_double), ("lr_final", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("w_mse", ctypes.c_double), ("w_res", ctypes.c_double),
                ("losses", ctypes.c_void_p)]


class hca_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * NKCLASS), ("ms", ctypes.c_double * NKCLASS)]

    def as_dict(self) -> Dict:
        return {name: {"launches": int(self.launches[i]), "ms": float(self.ms[i])}
                for i, name in enumerate(KCLASS_NAMES)}


EXPORTS = [
    "hca_config_default", "hca_create", "hca_create_batch", "hca_step", "hca_stage",
    "hca_read_fields", "hca_write_fields", "hca_read_states", "hca_write_states",
    "hca_set_step", "hca_get_stats", "hca_apply_operator", "hca_apply_preconditioner", "hca_philox_uniforms",
    "hca_get_launch_config",
    "hca_sync", "hca_get_shape", "hca_launch_count", "hca_profile_enable", "hca_get_profile",
    "hca_o2_residual_noalloc", "hca_save", "hca_load", "hca_destroy", "hca_status_string",
    "hca_net_param_count", "hca_net_create", "hca_net_set_params", "hca_net_get_params", "hca_net_forward",
    "hca_net_forward_x", "hca_net_read_activation", "hca_net_read_gradient", "hca_net_gradients_x", "hca_net_gradients", "hca_net_adam", "hca_net_train_step", "hca_train_warmstart", "hca_net_sync",
    "hca_net_destroy", "hca_set_warm_start_net",
]

NET_IN_CH = 16
NET_SCALE = 64.0


_lib = None


class HcaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.hca_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libhca.so (building it first if absent).  Raises if it cannot load."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libhca.so not built at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I32, I64, U32, U64, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
    cfgp = ctypes.POINTER(hca_config)
    sig = {
        "hca_config_default": (ctypes.c_int, [cfgp, I32, I32, I32]),
        "hca_create": (ctypes.c_int, [cfgp, P, P, P, I32, ctypes.POINTER(P)]),
        "hca_create_batch": (ctypes.c_int, [I32, cfgp, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                            I32, ctypes.POINTER(P)]),
        "hca_step": (ctypes.c_int, [P, I32]),
        "hca_stage": (ctypes.c_int, [P, U32]),
        "hca_read_fields": (ctypes.c_int, [P, I32, U32, P, SZ, I32]),
        "hca_write_fields": (ctypes.c_int, [P, I32, U32, P, SZ, I32]),
        "hca_read_states": (ctypes.c_int, [P, I32, P, SZ, I32]),
        "hca_write_states": (ctypes.c_int, [P, I32, P, SZ, I32]),
        "hca_set_step": (ctypes.c_int, [P, I64]),
        "hca_get_stats": (ctypes.c_int, [P, I32, ctypes.POINTER(hca_stats)]),
        "hca_apply_operator": (ctypes.c_int, [P, I32, I32, P, P, I32]),
        "hca_apply_preconditioner": (ctypes.c_int, [P, I32, I32, P, P, I32]),
        "hca_get_launch_config": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "hca_philox_uniforms": (ctypes.c_int, [U64, U64, I64, U32, U32, P, I32]),
        "hca_sync": (ctypes.c_int, [P]),
        "hca_get_shape": (ctypes.c_int, [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "hca_launch_count": (I64, [P]),
        "hca_profile_enable": (ctypes.c_int, [P, I32]),
        "hca_get_profile": (ctypes.c_int, [P, ctypes.POINTER(hca_profile)]),
        "hca_o2_residual_noalloc": (ctypes.c_int, [cfgp, P, P, P, ctypes.POINTER(ctypes.c_double), P]),
        "hca_save": (ctypes.c_int, [P, ctypes.c_char_p]),
        "hca_load": (ctypes.c_int, [ctypes.c_char_p, P, ctypes.POINTER(P)]),
        "hca_destroy": (None, [P]),
        "hca_status_string": (ctypes.c_char_p, [I32]),
        "hca_net_param_count": (ctypes.c_int, [ctypes.POINTER(I64)]),
        "hca_net_create": (ctypes.c_int, [I32, I32, I32, I32, P, ctypes.POINTER(P)]),
        "hca_net_set_params": (ctypes.c_int, [P, P, I32]),
        "hca_net_get_params": (ctypes.c_int, [P, P, I32]),
        "hca_net_forward": (ctypes.c_int, [P, cfgp, P, P, P, P, P]),
        "hca_net_forward_x": (ctypes.c_int, [P, P, P]),
        "hca_net_read_activation": (ctypes.c_int, [P, I32, P]),
        "hca_net_read_gradient": (ctypes.c_int, [P, I32, P]),
        "hca_net_gradients_x": (ctypes.c_int, [P, P, P, P, P]),
        "hca_net_adam": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "hca_net_gradients": (ctypes.c_int, [P, cfgp, P, P, P, P, ctypes.c_double, ctypes.c_double, P, P]),
        "hca_net_train_step": (ctypes.c_int, [P, cfgp, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, P]),
        "hca_train_warmstart": (ctypes.c_int, [P, cfgp, ctypes.POINTER(hca_train_cfg)]),
        "hca_net_sync": (ctypes.c_int, [P]),
        "hca_net_destroy": (ctypes.c_int, [P]),
        "hca_set_warm_start_net": (ctypes.c_int, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != HCA_OK:
        raise HcaError(rc, what)


# ------------------------------------------------------------ config ---
_ARRAY3 = {"D_G", "psi_G", "kappa_G", "uptake_G", "dose_peak", "plasma_decay", "kill_b", "pk_model", "epi_w"}


def make_config(nx: int, ny: int, nz: int, precision="f64", stream=None, **params) -> hca_config:
    """hca_config from the library defaults plus overrides (names as in hca.h)."""
    lib = load()
    cfg = hca_config()
    _check(lib.hca_config_default(ctypes.byref(cfg), nx, ny, nz), "hca_config_default")
    cfg.precision = HCA_FP32 if precision in ("f32", HCA_FP32) else HCA_FP64
    for k, v in params.items():
        if k in _ARRAY3:
            arr = getattr(cfg, k)
            vals = list(v)
            for i in range(min(3, len(vals))):
                arr[i] = vals[i]
        elif k == "seed":
            cfg.seed = int(v) & 0xFFFFFFFFFFFFFFFF
        elif hasattr(cfg, k):
            setattr(cfg, k, v)
        else:
            raise KeyError(f"unknown hca_config field {k!r}")
    if stream is not None:
        cfg.stream = ctypes.c_void_p(int(stream))
    return cfg


# ---------------------------------------------------------- buffers ---
def _ptr(buf):
    """(pointer, nbytes, on_device) for a numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("host buffers must be C-contiguous")
        return buf.ctypes.data, buf.nbytes, 0
    # torch tensor
    if not buf.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return buf.data_ptr(), buf.numel() * buf.element_size(), 1 if buf.is_cuda else 0


# --------------------------------------------------------------- API ---
def hca_config_default(nx, ny, nz) -> hca_config:
    return make_config(nx, ny, nz)


def hca_create(cfg: hca_config, p_cell, perf, p_vessel):
    lib = load()
    ptrs = [_ptr(m) for m in (p_cell, perf, p_vessel)]
    on_dev = ptrs[0][2]
    if any(p[2] != on_dev for p in ptrs):
        raise ValueError("maps must all be on the host or all on the device")
    n = cfg.nx * cfg.ny * cfg.nz
    for m, p in zip((p_cell, perf, p_vessel), ptrs):
        if p[1] < 4 * n:
            raise ValueError("map too small")
    h = ctypes.c_void_p()
    _check(lib.hca_create(ctypes.byref(cfg), ptrs[0][0], ptrs[1][0], ptrs[2][0], on_dev, ctypes.byref(h)),
           "hca_create")
    return h


def hca_create_batch(cfgs: Sequence[hca_config], p_cell, perf, p_vessel):
    lib = load()
    n = len(cfgs)
    arr = (hca_config * n)(*cfgs)
    pc = [_ptr(m) for m in p_cell]
    pf = [_ptr(m) for m in perf]
    pv = [_ptr(m) for m in p_vessel]
    on_dev = pc[0][2]
    mk = lambda lst: (ctypes.c_void_p * n)(*[p[0] for p in lst])
    h = ctypes.c_void_p()
    _check(lib.hca_create_batch(n, arr, mk(pc), mk(pf), mk(pv), on_dev, ctypes.byref(h)), "hca_create_batch")
    return h


def hca_step(h, n_steps: int = 1) -> int:
    return load().hca_step(h, n_steps)


def hca_stage(h, mask: int) -> int:
    return load().hca_stage(h, mask)


def hca_read_fields(h, rep: int, mask: int, dst) -> None:
    p, nb, dev = _ptr(dst)
    _check(load().hca_read_fields(h, rep, mask, p, nb, dev), "hca_read_fields")


def hca_write_fields(h, rep: int, mask: int, src) -> None:
    p, nb, dev = _ptr(src)
    _check(load().hca_write_fields(h, rep, mask, p, nb, dev), "hca_write_fields")


def hca_read_states(h, rep: int, dst) -> None:
    p, nb, dev = _ptr(dst)
    _check(load().hca_read_states(h, rep, p, nb, dev), "hca_read_states")


def hca_write_states(h, rep: int, src) -> None:
    p, nb, dev = _ptr(src)
    _check(load().hca_write_states(h, rep, p, nb, dev), "hca_write_states")


def hca_set_step(h, step: int) -> None:
    _check(load().hca_set_step(h, step), "hca_set_step")


def hca_get_stats(h, rep: int = 0) -> hca_stats:
    st = hca_stats()
    _check(load().hca_get_stats(h, rep, ctypes.byref(st)), "hca_get_stats")
    return st


def hca_apply_operator(h, rep: int, which: int, u, out) -> None:
    pu, nu, du = _ptr(u)
    po, no, do = _ptr(out)
    if du != do or nu != no:
        raise ValueError("u and out must match in size and location")
    _check(load().hca_apply_operator(h, rep, which, pu, po, du), "hca_apply_operator")


def hca_get_launch_config(h):
    t, r = ctypes.c_int32(), ctypes.c_int32()
    _check(load().hca_get_launch_config(h, ctypes.byref(t), ctypes.byref(r)), "hca_get_launch_config")
    return t.value, r.value


def hca_apply_preconditioner(h, rep: int, which: int, r, z) -> None:
    pr, nr, dr = _ptr(r)
    pz, nz, dz = _ptr(z)
    if dr != dz or nr != nz:
        raise ValueError("r and z must match in size and location")
    _check(load().hca_apply_preconditioner(h, rep, which, pr, pz, dr), "hca_apply_preconditioner")


def hca_philox_uniforms(seed: int, site_begin: int, n: int, step: int, purpose: int, dst=None):
    if dst is None:
        dst = np.empty(n, dtype=np.float32)
    p, nb, dev = _ptr(dst)
    if nb < 4 * n:
        raise ValueError("dst too small")
    _check(load().hca_philox_uniforms(seed & 0xFFFFFFFFFFFFFFFF, site_begin, n, step, purpose, p, dev),
           "hca_philox_uniforms")
    return dst


def hca_sync(h) -> None:
    _check(load().hca_sync(h), "hca_sync")


def hca_launch_count(h) -> int:
    return int(load().hca_launch_count(h))


def hca_profile_enable(h, enable: bool = True) -> None:
    _check(load().hca_profile_enable(h, 1 if enable else 0), "hca_profile_enable")


def hca_get_profile(h) -> Dict:
    out = hca_profile()
    _check(load().hca_get_profile(h, ctypes.byref(out)), "hca_get_profile")
    return out.as_dict()


def hca_o2_residual_noalloc(cfg: hca_config, state, K_prev, K, stream=None) -> float:
    """||b - A(K_prev) K|| / ||b|| on caller-owned device tensors, with no device
    allocation (for callers that may not allocate; see include/hca.h)."""
    ptrs = [_ptr(t) for t in (state, K_prev, K)]
    if not all(p[2] for p in ptrs):
        raise ValueError("state, K_prev and K must be device tensors")
    n = cfg.nx * cfg.ny * cfg.nz
    if ptrs[0][1] < n or ptrs[1][1] < 8 * n or ptrs[2][1] < 8 * n:
        raise ValueError("arrays too small for the lattice")
    out = ctypes.c_double()
    _check(load().hca_o2_residual_noalloc(ctypes.byref(cfg), ptrs[0][0], ptrs[1][0], ptrs[2][0], ctypes.byref(out),
                                          ctypes.c_void_p(int(stream) if stream else 0)), "hca_o2_residual_noalloc")
    return out.value


def hca_destroy(h) -> None:
    if h:
        load().hca_destroy(h)


def hca_save(h, path: str) -> None:
    _check(load().hca_save(h, os.fsencode(path)), "hca_save")


def hca_load(path: str, stream=None):
    h = ctypes.c_void_p()
    _check(load().hca_load(os.fsencode(path), ctypes.c_void_p(int(stream)) if stream is not None else None,
                           ctypes.byref(h)), "hca_load")
    return h


def checkpoint_configs(path: str):
    """The configurations stored in a checkpoint file (its header is read
    here; see hca_save for the format)."""
    with open(path, "rb") as f:
        head = f.read(40)
        if len(head) != 40 or head[:8] != b"HCACKPT1":
            raise ValueError("not a checkpoint file")
        version, csize, n, _prec = struct.unpack("<4i", head[8:24])
        if version != 1 or csize != ctypes.sizeof(hca_config):
            raise ValueError("checkpoint of another ABI")
        cfgs = []
        for _ in range(n):
            cfg = hca_config()
            ctypes.memmove(ctypes.byref(cfg), f.read(csize), csize)
            cfgs.append(cfg)
    return cfgs


# ------------------------------------------- learned warm start (net) ---
def _dev(t, what, nbytes=None):
    p, nb, on_dev = _ptr(t)
    if not on_dev:
        raise ValueError(f"{what} must be a device tensor")
    if nbytes is not None and nb < nbytes:
        raise ValueError(f"{what} too small ({nb} < {nbytes} bytes)")
    return p


def hca_net_param_count() -> int:
    n = ctypes.c_int64()
    _check(load().hca_net_param_count(ctypes.byref(n)), "hca_net_param_count")
    return n.value


def hca_net_create(D: int, H: int, W: int, trainable: bool = False, stream=None):
    h = ctypes.c_void_p()
    _check(load().hca_net_create(D, H, W, 1 if trainable else 0, ctypes.c_void_p(int(stream) if stream else 0),
                                 ctypes.byref(h)), "hca_net_create")
    return h


def hca_net_set_params(net, params) -> None:
    n = hca_net_param_count()
    if isinstance(params, np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
    p, nb, on_dev = _ptr(params)
    if nb < 4 * n:
        raise ValueError("parameter array too small")
    _check(load().hca_net_set_params(net, p, on_dev), "hca_net_set_params")


def hca_net_get_params(net) -> np.ndarray:
    out = np.empty(hca_net_param_count(), dtype=np.float32)
    _check(load().hca_net_get_params(net, out.ctypes.data, 0), "hca_net_get_params")
    return out


def hca_net_forward(net, cfg: hca_config, state, perf, K_prev, out, x_out=None) -> None:
    n = cfg.nx * cfg.ny * cfg.nz
    _check(load().hca_net_forward(net, ctypes.byref(cfg), _dev(state, "state", n), _dev(perf, "perf", 4 * n),
                                  _dev(K_prev, "K_prev", 4 * n), _dev(out, "out", 4 * n),
                                  _dev(x_out, "x_out", 32 * n) if x_out is not None else None), "hca_net_forward")


def hca_net_forward_x(net, x, out) -> None:
    _check(load().hca_net_forward_x(net, _dev(x, "x"), _dev(out, "out")), "hca_net_forward_x")


# stored activations: (name, level, channels) in hca_net_read_activation order
NET_ACTIVATIONS = (("x", 0, 16), ("e0", 0, 16), ("p0", 1, 16), ("e1", 1, 32), ("p1", 2, 32), ("e2", 2, 64),
                   ("p2", 3, 64), ("e3", 3, 64), ("d2", 2, 64), ("d1", 1, 32), ("d0", 0, 16))


def hca_net_read_activation(net, which: int, dst) -> None:
    _check(load().hca_net_read_activation(net, which, _dev(dst, "dst")), "hca_net_read_activation")


def hca_net_read_gradient(net, which: int, dst) -> None:
    _check(load().hca_net_read_gradient(net, which, _dev(dst, "dst")), "hca_net_read_gradient")


def hca_net_gradients_x(net, x, target, grads=None, loss=None) -> None:
    _check(load().hca_net_gradients_x(net, _dev(x, "x"), _dev(target, "target"),
                                      _dev(grads, "grads", 4 * hca_net_param_count()) if grads is not None else None,
                                      _dev(loss, "loss", 4) if loss is not None else None), "hca_net_gradients_x")


def hca_net_adam(net, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    _check(load().hca_net_adam(net, lr, beta1, beta2, eps), "hca_net_adam")


def hca_net_gradients(net, cfg: hca_config, state, perf, K_prev, K_new, w_mse: float = 1.0, w_res: float = 0.0,
                      grads=None, loss=None) -> None:
    n = cfg.nx * cfg.ny * cfg.nz
    _check(load().hca_net_gradients(net, ctypes.byref(cfg), _dev(state, "state", n), _dev(perf, "perf", 4 * n),
                                    _dev(K_prev, "K_prev", 4 * n), _dev(K_new, "K_new", 4 * n), w_mse, w_res,
                                    _dev(grads, "grads", 4 * hca_net_param_count()) if grads is not None else None,
                                    _dev(loss, "loss", 4) if loss is not None else None), "hca_net_gradients")


def hca_net_train_step(net, cfg: hca_config, state, perf, K_prev, K_new, lr: float, loss=None,
                       w_mse: float = 1.0, w_res: float = 0.0) -> None:
    n = cfg.nx * cfg.ny * cfg.nz
    _check(load().hca_net_train_step(net, ctypes.byref(cfg), _dev(state, "state", n), _dev(perf, "perf", 4 * n),
                                     _dev(K_prev, "K_prev", 4 * n), _dev(K_new, "K_new", 4 * n), w_mse, w_res, lr,
                                     _dev(loss, "loss", 4) if loss is not None else None), "hca_net_train_step")


def hca_train_warmstart(net, cfg: hca_config, states, perfs, K_prevs, K_news, iters: int, lr: float,
                        lr_final: float, seed: int = 0, w_mse: float = 1.0, w_res: float = 0.0, losses=None) -> None:
    """The whole training run in one library call (sequences of device tensors,
    one entry per sample; see include/hca.h)."""
    n = cfg.nx * cfg.ny * cfg.nz
    k = len(states)
    if not (len(perfs) == len(K_prevs) == len(K_news) == k):
        raise ValueError("one state, perf, K_prev and K_new per sample")
    arr = lambda ts, name, nb: (ctypes.c_void_p * k)(*[_dev(t, name, nb) for t in ts])
    tc = hca_train_cfg()
    tc.struct_size = ctypes.sizeof(hca_train_cfg)
    tc.n_samples = k
    keep = [arr(states, "state", n), arr(perfs, "perf", 4 * n), arr(K_prevs, "K_prev", 4 * n),
            arr(K_news, "K_new", 4 * n)]
    tc.state, tc.perf, tc.K_prev, tc.K_new = [ctypes.cast(a, ctypes.POINTER(ctypes.c_void_p)) for a in keep]
    tc.iters, tc.lr, tc.lr_final, tc.seed = iters, lr, lr_final, seed & 0xFFFFFFFFFFFFFFFF
    tc.w_mse, tc.w_res = w_mse, w_res
    tc.losses = _dev(losses, "losses", 4 * iters) if losses is not None else None
    _check(load().hca_train_warmstart(net, ctypes.byref(cfg), ctypes.byref(tc)), "hca_train_warmstart")


def hca_net_sync(net) -> None:
    _check(load().hca_net_sync(net), "hca_net_sync")


def hca_net_destroy(net) -> None:
    if net:
        load().hca_net_destroy(net)


def hca_set_warm_start_net(h, net) -> None:
    _check(load().hca_set_warm_start_net(h, net if net else None), "hca_set_warm_start_net")


class Net:
    """The warm-start network for one D x H x W lattice (device tensors in and out)."""

    def __init__(self, D: int, H: int, W: int, trainable: bool = False, stream=None):
        self.shape = (D, H, W)
        self.handle = hca_net_create(D, H, W, trainable, stream)

    def set_params(self, params) -> None:
        hca_net_set_params(self.handle, params)

    def params(self) -> np.ndarray:
        return hca_net_get_params(self.handle)

    def close(self) -> None:
        if self.handle:
            hca_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ convenience ---
class Sim:
    """One handle (one replicate or a batch) with numpy-friendly helpers."""

    def __init__(self, cfgs, maps, batch: bool = False):
        if batch:
            self.cfgs = list(cfgs)
            self.handle = hca_create_batch(self.cfgs, [m[0] for m in maps], [m[1] for m in maps],
                                           [m[2] for m in maps])
        else:
            self.cfgs = [cfgs]
            self.handle = hca_create(cfgs, *maps)
        self.fp64 = self.cfgs[0].precision == HCA_FP64
        self.dtype = np.float64 if self.fp64 else np.float32

    @classmethod
    def create(cls, nx, ny, nz, p_cell, perf, p_vessel, precision="f64", **params):
        return cls(make_config(nx, ny, nz, precision=precision, **params), (p_cell, perf, p_vessel))

    def shape(self, rep: int = 0):
        c = self.cfgs[rep]
        return (c.nz, c.ny, c.nx)

    def step(self, n: int = 1, allow_noconv: bool = False) -> int:
        rc = hca_step(self.handle, n)
        if rc != HCA_OK and not (allow_noconv and rc == HCA_ERR_NOCONV):
            raise HcaError(rc, "hca_step")
        return rc

    def stage(self, mask: int, allow_noconv: bool = False) -> int:
        rc = hca_stage(self.handle, mask)
        if rc != HCA_OK and not (allow_noconv and rc == HCA_ERR_NOCONV):
            raise HcaError(rc, "hca_stage")
        return rc

    def field(self, bit: int, rep: int = 0) -> np.ndarray:
        out = np.empty(self.shape(rep), dtype=self.dtype)
        hca_read_fields(self.handle, rep, bit, out)
        return out

    def set_field(self, bit: int, values, rep: int = 0) -> None:
        arr = np.ascontiguousarray(np.asarray(values, dtype=self.dtype).reshape(self.shape(rep)))
        hca_write_fields(self.handle, rep, bit, arr)

    def states(self, rep: int = 0) -> np.ndarray:
        out = np.empty(self.shape(rep), dtype=np.uint8)
        hca_read_states(self.handle, rep, out)
        return out

    def set_states(self, values, rep: int = 0) -> None:
        hca_write_states(self.handle, rep, np.ascontiguousarray(np.asarray(values, dtype=np.uint8)))

    def stats(self, rep: int = 0) -> Dict:
        return hca_get_stats(self.handle, rep).as_dict()

    def apply_operator(self, which: int, u, rep: int = 0) -> np.ndarray:
        u = np.ascontiguousarray(np.asarray(u, dtype=self.dtype).reshape(self.shape(rep)))
        out = np.empty_like(u)
        hca_apply_operator(self.handle, rep, which, u, out)
        return out

    def apply_preconditioner(self, which: int, r, rep: int = 0) -> np.ndarray:
        r = np.ascontiguousarray(np.asarray(r, dtype=self.dtype).reshape(self.shape(rep)))
        z = np.empty_like(r)
        hca_apply_preconditioner(self.handle, rep, which, r, z)
        return z

    def set_step(self, n: int) -> None:
        hca_set_step(self.handle, n)

    def launches(self) -> int:
        return hca_launch_count(self.handle)

    def save(self, path: str) -> None:
        hca_save(self.handle, path)

    @classmethod
    def load(cls, path: str, stream=None) -> "Sim":
        sim = cls.__new__(cls)
        sim.cfgs = checkpoint_configs(path)
        sim.handle = hca_load(path, stream)
        sim.fp64 = sim.cfgs[0].precision == HCA_FP64
        sim.dtype = np.float64 if sim.fp64 else np.float32
        return sim

    def set_warm_start_net(self, net) -> None:
        hca_set_warm_start_net(self.handle, net.handle if isinstance(net, Net) else net)

    def close(self) -> None:
        if self.handle:
            hca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
