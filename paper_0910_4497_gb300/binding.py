"""ctypes binding of the C ABI in include/tb.h.

Argument marshalling only: every function below checks tensor dtype, device
and contiguity, then forwards raw device pointers, sizes and the current CUDA
stream to the function of the same name in libtb.so.  There is no CPU path: if
the library is missing, importing this module raises.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtb.so")

TB_OK = 0
STATUS_NAMES = {0: "TB_OK", 1: "TB_ERR_INVALID_ARG", 2: "TB_ERR_CUDA", 3: "TB_ERR_NOMEM",
                4: "TB_ERR_CAPACITY", 5: "TB_ERR_NONFINITE", 6: "TB_ERR_BREAKDOWN",
                7: "TB_ERR_NO_CONVERGENCE", 8: "TB_ERR_TIMEOUT", 9: "TB_ERR_NOT_RESERVED"}
TB_PREC_FP64 = 0
TB_PREC_MIXED = 1
TB_PREC_BF16 = 2
PRECISIONS = {"fp64": TB_PREC_FP64, "mixed": TB_PREC_MIXED, "bf16": TB_PREC_BF16}
SCHEDULES = {"auto": 0, "persistent": 1, "separate": 2, "persistent_largest_first": 3,
             "bucketed": 4}
SCHEDULE_NAMES = {v: k for k, v in SCHEDULES.items()}
TUNE_MAX_BUCKETS = 4
TUNE_BINS = 128

EXPORTS = ["tb_params_default", "tb_ctx_create", "tb_ctx_destroy", "tb_ctx_reserve",
           "tb_ctx_workspace_bytes", "tb_get_status", "tb_build_neighbors",
           "tb_assemble_H", "tb_krylov_density", "tb_find_mu", "tb_forces", "tb_md_step",
           "tb_profile_enable", "tb_profile_read", "tb_find_mu_static",
           "tb_virial", "tb_ctx_reserve_local", "tb_local_forward", "tb_local_gradient",
           "tb_group_atoms", "tb_krylov_density_grouped", "tb_ctx_kernels_per_evaluation",
           "tb_npt_berendsen", "tb_autotune", "tb_version"]


class TBParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("Es", "Ep", "Vss", "Vsp", "Vpps", "Vppp", "r0", "n", "nc", "rc",
                 "phi0", "d0", "m", "mc", "dc", "r1", "rm", "kT", "Rc", "defl_tol",
                 "mu_tol")] + \
              [(k, ctypes.c_int) for k in
               ("r", "prec", "max_hnbr", "max_cluster", "reorth_passes", "mu_max_iter")] + \
              [("timeout_cycles", ctypes.c_longlong), ("reorth_every", ctypes.c_int),
               ("group_m", ctypes.c_int), ("max_union", ctypes.c_int),
               ("schedule", ctypes.c_int)]


class TBTuneReport(ctypes.Structure):
    _fields_ = [("bin_width", ctypes.c_int), ("n_bins", ctypes.c_int),
                ("hist", ctypes.c_int * TUNE_BINS), ("schedule", ctypes.c_int),
                ("ms_persistent", ctypes.c_float), ("ms_persistent_largest_first", ctypes.c_float),
                ("ms_separate", ctypes.c_float), ("ms_bucketed", ctypes.c_float),
                ("persistent_records_per_slot", ctypes.c_int),
                ("persistent_ctas_per_sm", ctypes.c_int),
                ("n_buckets", ctypes.c_int),
                ("bucket_hi", ctypes.c_int * TUNE_MAX_BUCKETS),
                ("bucket_count", ctypes.c_int * TUNE_MAX_BUCKETS),
                ("bucket_records_per_slot", ctypes.c_int * TUNE_MAX_BUCKETS),
                ("bucket_ctas_per_sm", ctypes.c_int * TUNE_MAX_BUCKETS),
                ("bucket_ms", ctypes.c_float * TUNE_MAX_BUCKETS)]


class TBError(RuntimeError):
    def __init__(self, fn, code, info=None):
        self.code = code
        self.info = info
        msg = f"{fn} -> {STATUS_NAMES.get(code, code)}"
        if info is not None:
            msg += f" (info {info})"
        super().__init__(msg)


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libtb.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "tb_params_default": [ctypes.POINTER(TBParams)],
        "tb_ctx_create": [ctypes.POINTER(P), ctypes.POINTER(TBParams)],
        "tb_ctx_destroy": [P],
        "tb_ctx_reserve": [P, I],
        "tb_ctx_workspace_bytes": [P, ctypes.POINTER(ctypes.c_size_t)],
        "tb_get_status": [P, ctypes.POINTER(I), ctypes.POINTER(I), VP],
        "tb_build_neighbors": [P, I, VP, D, VP, VP, VP, VP, VP],
        "tb_assemble_H": [P, I, VP, D, VP, VP, VP, VP, VP, VP],
        "tb_krylov_density": [P, I, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "tb_find_mu": [P, I, VP, VP, VP, D, VP, VP, VP, VP],
        "tb_forces": [P, I, VP, D, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "tb_md_step": [P, I, VP, VP, VP, D, D, D, VP, VP],
        "tb_profile_enable": [P, I],
        "tb_profile_read": [P, ctypes.POINTER(ctypes.c_float)],
        "tb_find_mu_static": [I, I, VP, VP, D, D, D, I, VP, VP, VP, VP, VP],
        "tb_virial": [P, I, VP, D, VP, VP, VP, VP, VP],
        "tb_npt_berendsen": [P, I, VP, VP, D, VP, VP, D, D, D, D, D, D, VP, VP, VP],
        "tb_ctx_reserve_local": [P, I],
        "tb_local_forward": [P, I, VP, D, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "tb_local_gradient": [P, I, VP, D, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "tb_group_atoms": [P, I, VP, D, VP, VP, VP],
        "tb_ctx_kernels_per_evaluation": [P, I, D, ctypes.POINTER(I)],
        "tb_krylov_density_grouped": [P, I, I, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "tb_autotune": [P, I, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, ctypes.POINTER(TBTuneReport), VP],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.tb_version.argtypes = []
    lib.tb_version.restype = ctypes.c_char_p
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(fn, code):
    if code != TB_OK:
        raise TBError(fn, code)


def _ptr(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(p, prec):
    """tb_params from a dict of model constants plus kT, Rc, r, caps."""
    tp = TBParams()
    _check("tb_params_default", lib().tb_params_default(ctypes.byref(tp)))
    for k in ("Es", "Ep", "Vss", "Vsp", "Vpps", "Vppp", "r0", "n", "nc", "rc", "phi0",
              "d0", "m", "mc", "dc", "r1", "rm", "kT", "Rc"):
        setattr(tp, k, float(p[k]))
    tp.r = int(p["r"])
    tp.max_hnbr = int(p.get("max_hnbr", 32))
    tp.max_cluster = int(p.get("max_cluster", 128))
    tp.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    tp.defl_tol = float(p.get("defl_tol", 1e-9 if tp.prec == TB_PREC_FP64 else 1e-4))
    tp.reorth_passes = int(p.get("reorth_passes", 2))
    tp.reorth_every = int(p.get("reorth_every", 1))
    tp.mu_tol = float(p.get("mu_tol", 1e-12))
    tp.mu_max_iter = int(p.get("mu_max_iter", 100))
    tp.group_m = int(p.get("group_m", 1))
    tp.max_union = int(p.get("max_union", 0))
    sched = p.get("schedule", "auto")
    tp.schedule = SCHEDULES[sched] if isinstance(sched, str) else int(sched)
    if "timeout_cycles" in p:
        tp.timeout_cycles = int(p["timeout_cycles"])
    return tp


# ---------------------------------------------------------------- same-name calls

def tb_ctx_create(params):
    h = ctypes.c_void_p()
    _check("tb_ctx_create", lib().tb_ctx_create(ctypes.byref(h), ctypes.byref(params)))
    return h


def tb_ctx_destroy(ctx):
    _check("tb_ctx_destroy", lib().tb_ctx_destroy(ctx))


def tb_ctx_reserve(ctx, n_atoms):
    _check("tb_ctx_reserve", lib().tb_ctx_reserve(ctx, int(n_atoms)))


def tb_ctx_workspace_bytes(ctx):
    b = ctypes.c_size_t()
    _check("tb_ctx_workspace_bytes", lib().tb_ctx_workspace_bytes(ctx, ctypes.byref(b)))
    return b.value


def tb_get_status(ctx, stream=None):
    code, info = ctypes.c_int(), ctypes.c_int()
    _check("tb_get_status", lib().tb_get_status(ctx, ctypes.byref(code), ctypes.byref(info),
                                                 _stream(stream)))
    return code.value, info.value


def tb_build_neighbors(ctx, n, pos, L, h_off, h_idx, c_off, c_idx, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_build_neighbors", lib().tb_build_neighbors(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(h_off, i32, "h_off"),
        _ptr(h_idx, i32, "h_idx"), _ptr(c_off, i32, "c_off"), _ptr(c_idx, i32, "c_idx"),
        _stream(stream)))


def tb_assemble_H(ctx, n, pos, L, h_off, h_idx, Hblk, dHblk, Hsk=None, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_assemble_H", lib().tb_assemble_H(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(h_off, i32, "h_off"),
        _ptr(h_idx, i32, "h_idx"), _ptr(Hblk, f64, "Hblk"), _ptr(dHblk, f64, "dHblk"),
        _ptr(Hsk, torch.float32, "Hsk"), _stream(stream)))


def tb_krylov_density(ctx, n, c_off, c_idx, h_off, h_idx, Hblk, Hsk, lam, S, P, kdim,
                      stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_krylov_density", lib().tb_krylov_density(
        ctx, n, _ptr(c_off, i32, "c_off"), _ptr(c_idx, i32, "c_idx"),
        _ptr(h_off, i32, "h_off"), _ptr(h_idx, i32, "h_idx"), _ptr(Hblk, f64, "Hblk"),
        _ptr(Hsk, torch.float32, "Hsk"), _ptr(lam, f64, "lambda"),
        _ptr(S, f64, "S"), _ptr(P, f64, "P"), _ptr(kdim, i32, "kdim"), _stream(stream)))


def tb_ctx_kernels_per_evaluation(ctx, n, L):
    k = ctypes.c_int()
    _check("tb_ctx_kernels_per_evaluation",
           lib().tb_ctx_kernels_per_evaluation(ctx, int(n), float(L), ctypes.byref(k)))
    return k.value


def tb_group_atoms(ctx, n, pos, L, g_off, g_idx, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_group_atoms", lib().tb_group_atoms(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(g_off, i32, "g_off"),
        _ptr(g_idx, i32, "g_idx"), _stream(stream)))


def tb_krylov_density_grouped(ctx, n, n_groups, g_off, g_idx, c_off, c_idx, h_off, h_idx,
                              Hblk, Hsk, lam, S, P, kdim, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_krylov_density_grouped", lib().tb_krylov_density_grouped(
        ctx, n, int(n_groups), _ptr(g_off, i32, "g_off"), _ptr(g_idx, i32, "g_idx"),
        _ptr(c_off, i32, "c_off"), _ptr(c_idx, i32, "c_idx"),
        _ptr(h_off, i32, "h_off"), _ptr(h_idx, i32, "h_idx"), _ptr(Hblk, f64, "Hblk"),
        _ptr(Hsk, torch.float32, "Hsk"), _ptr(lam, f64, "lambda"),
        _ptr(S, f64, "S"), _ptr(P, f64, "P"), _ptr(kdim, i32, "kdim"), _stream(stream)))


def tb_autotune(ctx, n, c_off, c_idx, h_off, h_idx, Hblk, Hsk, lam, S, P, kdim, stream=None):
    """Times the launch plans of the mixed Krylov stage on these lists and keeps
    the fastest in the context; returns the report as a dict."""
    i32, f64 = torch.int32, torch.float64
    r = TBTuneReport()
    _check("tb_autotune", lib().tb_autotune(
        ctx, n, _ptr(c_off, i32, "c_off"), _ptr(c_idx, i32, "c_idx"), _ptr(h_off, i32, "h_off"),
        _ptr(h_idx, i32, "h_idx"), _ptr(Hblk, f64, "Hblk"), _ptr(Hsk, torch.float32, "Hsk"),
        _ptr(lam, f64, "lambda"), _ptr(S, f64, "S"), _ptr(P, f64, "P"), _ptr(kdim, i32, "kdim"),
        ctypes.byref(r), _stream(stream)))
    nb = r.n_buckets
    inf = 1e29
    return {"histogram": {"bin_width": r.bin_width,
                          "counts": list(r.hist[:r.n_bins])},
            "schedule": SCHEDULE_NAMES.get(r.schedule, r.schedule),
            "ms": {k: (v if v < inf else None) for k, v in
                   (("persistent", r.ms_persistent),
                    ("persistent_largest_first", r.ms_persistent_largest_first),
                    ("separate", r.ms_separate), ("bucketed", r.ms_bucketed))},
            "persistent_tile": {"records_per_slot_in_smem": r.persistent_records_per_slot,
                                "ctas_per_sm": r.persistent_ctas_per_sm},
            "buckets": [{"sizes_up_to": r.bucket_hi[b], "targets": r.bucket_count[b],
                         "records_per_slot_in_smem": r.bucket_records_per_slot[b],
                         "ctas_per_sm": r.bucket_ctas_per_sm[b], "ms": r.bucket_ms[b]}
                        for b in range(nb)]}


def tb_find_mu(ctx, n, lam, S, kdim, n_electrons, mu_guess, mu, n_count=None, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_find_mu", lib().tb_find_mu(
        ctx, n, _ptr(lam, f64, "lambda"), _ptr(S, f64, "S"), _ptr(kdim, i32, "kdim"),
        float(n_electrons), _ptr(mu_guess, f64, "mu_guess"), _ptr(mu, f64, "mu"),
        _ptr(n_count, f64, "n_count"), _stream(stream)))


def tb_forces(ctx, n, pos, L, h_off, h_idx, dHblk, lam, S, P, kdim, mu, F, energies,
              stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_forces", lib().tb_forces(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(h_off, i32, "h_off"),
        _ptr(h_idx, i32, "h_idx"), _ptr(dHblk, f64, "dHblk"), _ptr(lam, f64, "lambda"),
        _ptr(S, f64, "S"), _ptr(P, f64, "P"), _ptr(kdim, i32, "kdim"), _ptr(mu, f64, "mu"),
        _ptr(F, f64, "F"), _ptr(energies, f64, "energies"), _stream(stream)))


def tb_md_step(ctx, n, pos, vel, F, L, dt_fs, mass_amu, energies, stream=None):
    f64 = torch.float64
    _check("tb_md_step", lib().tb_md_step(
        ctx, n, _ptr(pos, f64, "pos"), _ptr(vel, f64, "vel"), _ptr(F, f64, "F"), float(L),
        float(dt_fs), float(mass_amu), _ptr(energies, f64, "energies"), _stream(stream)))


STAGES = ("lists", "assemble", "krylov", "eig", "mu", "forces", "grouping")


def tb_profile_enable(ctx, enable=True):
    _check("tb_profile_enable", lib().tb_profile_enable(ctx, 1 if enable else 0))


def tb_profile_read(ctx):
    ms = (ctypes.c_float * 7)()
    _check("tb_profile_read", lib().tb_profile_read(ctx, ms))
    return dict(zip(STAGES, list(ms)))


def tb_find_mu_static(n, r, lam, S, kT, n_electrons, mu_tol, max_iter, mu_guess, mu,
                      n_count, status, stream=None):
    """Allocation-free mu search (no context); status is a device int32[2]."""
    i32, f64 = torch.int32, torch.float64
    _check("tb_find_mu_static", lib().tb_find_mu_static(
        int(n), int(r), _ptr(lam, f64, "lambda"), _ptr(S, f64, "S"), float(kT),
        float(n_electrons), float(mu_tol), int(max_iter), _ptr(mu_guess, f64, "mu_guess"),
        _ptr(mu, f64, "mu"), _ptr(n_count, f64, "n_count"), _ptr(status, i32, "status"),
        _stream(stream)))


def tb_virial(ctx, n, pos, L, h_off, h_idx, W, pressure=None, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_virial", lib().tb_virial(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(h_off, i32, "h_off"),
        _ptr(h_idx, i32, "h_idx"), _ptr(W, f64, "W"), _ptr(pressure, f64, "pressure"),
        _stream(stream)))


def tb_npt_berendsen(ctx, n, pos, vel, L, W, energies, T0, P0, dt_fs, tau_T_fs, tau_P_fs,
                     beta, L_new, state, stream=None):
    f64 = torch.float64
    _check("tb_npt_berendsen", lib().tb_npt_berendsen(
        ctx, n, _ptr(pos, f64, "pos"), _ptr(vel, f64, "vel"), float(L), _ptr(W, f64, "W"),
        _ptr(energies, f64, "energies"), float(T0), float(P0), float(dt_fs), float(tau_T_fs),
        float(tau_P_fs), float(beta), _ptr(L_new, f64, "L_new"), _ptr(state, f64, "state"),
        _stream(stream)))


def tb_ctx_reserve_local(ctx, n_atoms):
    _check("tb_ctx_reserve_local", lib().tb_ctx_reserve_local(ctx, int(n_atoms)))


def _zstore(Z):
    if Z is None:
        return None
    if Z.dtype not in (torch.float32, torch.float64):
        raise TypeError("Zstore: expected float32 or float64")
    return _ptr(Z, Z.dtype, "Zstore")


def tb_local_forward(ctx, n, pos, L, c_off, c_idx, h_off, h_idx, Hblk, lam, S, kdim, Zstore,
                     mu, energies, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_local_forward", lib().tb_local_forward(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(c_off, i32, "c_off"),
        _ptr(c_idx, i32, "c_idx"), _ptr(h_off, i32, "h_off"), _ptr(h_idx, i32, "h_idx"),
        _ptr(Hblk, f64, "Hblk"), _ptr(lam, f64, "lambda"), _ptr(S, f64, "S"),
        _ptr(kdim, i32, "kdim"), _zstore(Zstore), _ptr(mu, f64, "mu"),
        _ptr(energies, f64, "energies"), _stream(stream)))


def tb_local_gradient(ctx, n, pos, L, c_off, c_idx, h_off, h_idx, Hblk, dHblk, lam, S, Zstore,
                      mu, F, stream=None):
    i32, f64 = torch.int32, torch.float64
    _check("tb_local_gradient", lib().tb_local_gradient(
        ctx, n, _ptr(pos, f64, "pos"), float(L), _ptr(c_off, i32, "c_off"),
        _ptr(c_idx, i32, "c_idx"), _ptr(h_off, i32, "h_off"), _ptr(h_idx, i32, "h_idx"),
        _ptr(Hblk, f64, "Hblk"), _ptr(dHblk, f64, "dHblk"), _ptr(lam, f64, "lambda"),
        _ptr(S, f64, "S"), _zstore(Zstore), _ptr(mu, f64, "mu"), _ptr(F, f64, "F"),
        _stream(stream)))


def tb_version():
    return lib().tb_version().decode()
