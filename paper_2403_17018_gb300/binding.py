"""ctypes binding of libhenry (include/henry.h): argument marshalling only.

Every computation runs in the CUDA library; torch supplies device memory and
streams. There is no CPU fallback: if libhenry.so cannot be loaded, calls
raise. Names follow the C ABI.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhenry.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "henry.h")

NQ = 22
QOI_NAMES = ("Q_S", "salt_mass", "toe", "c_x3", "c_x9", "c_x15")
PREC_FP64 = 0
PREC_FP32_MG = 1
LOOP_HOST = 0
LOOP_GRAPH = 1
DISC_CELL = 0
DISC_VERTEX = 1
S_MAXIT, S_NONFINITE, S_BADINPUT, S_STALL = 1, 2, 4, 8
ERRORS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -5: "unsupported grid"}


class HenryError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class HenryConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("rho0", "rho1", "mu", "g", "D", "K0", "phi0", "q0", "Lx", "Ly", "T")] + \
               [(n, ctypes.c_int) for n in ("nx0", "ny0", "nt0", "nlevels", "n_xi", "precision",
                                             "loop_mode")] + \
               [("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("guess_extrapolation", ctypes.c_int),
                ("newton_stag_tol", ctypes.c_double), ("mg_fusion", ctypes.c_int),
                ("mg_cluster_cells", ctypes.c_int), ("mg_small_cells", ctypes.c_int),
                ("jac_lag", ctypes.c_int), ("field_model", ctypes.c_int),
                ("krylov_iters", ctypes.c_int), ("adjoint_rtol", ctypes.c_double),
                ("res_rows", ctypes.c_int), ("discretisation", ctypes.c_int),
                ("mg_tb_cells", ctypes.c_int), ("jac_keep", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class HenrySchedule(ctypes.Structure):
    """Multigrid schedule of one MLMC level (henry_schedule)."""
    _fields_ = [(n, ctypes.c_int) for n in ("vcycles", "nu1", "nu2", "mg_small_cells", "jac_lag",
                                             "res_rows", "mg_tb_cells", "jac_keep")]


class HenryLevelBatch(ctypes.Structure):
    """One level's pairs for henry_sample_levels (henry_level_batch)."""
    _fields_ = [("level", ctypes.c_int), ("B", ctypes.c_int), ("xi", ctypes.c_void_p),
                ("q_fine", ctypes.c_void_p), ("q_coarse", ctypes.c_void_p),
                ("c_fine", ctypes.c_void_p), ("c_coarse", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class LevelStats(ctypes.Structure):
    """Running per-QoI statistics of one MLMC level (henry_level_stats)."""
    _fields_ = [("n", ctypes.c_int64), ("mean_f", ctypes.c_double * NQ),
                ("m2_f", ctypes.c_double * NQ), ("mean_d", ctypes.c_double * NQ),
                ("m2_d", ctypes.c_double * NQ)]

    def numpy(self):
        n = self.n
        den = max(n - 1, 1)
        return {"n": n, "mean_f": np.array(self.mean_f[:]), "var_f": np.array(self.m2_f[:]) / den,
                "mean_d": np.array(self.mean_d[:]), "var_d": np.array(self.m2_d[:]) / den}


_lib = None


def load():
    """Load libhenry.so (built by paper_2403_17018_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2403_17018_gb300.build.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    cfgp = ctypes.POINTER(HenryConfig)
    sig = {
        "henry_default_config": (I, [cfgp]),
        "henry_create_levels": (I, [cfgp, ctypes.POINTER(P)]),
        "henry_destroy": (None, [P]),
        "henry_solve": (I, [P, I, V, V, I, V, V, V, V, V, V]),
        "henry_sample_pairs": (I, [P, I, V, I, V, V, V, V, V, V]),
        "henry_solve_series": (I, [P, I, V, V, I, I, V, V, V, V]),
        "henry_set_schedule": (I, [P, I, ctypes.POINTER(HenrySchedule)]),
        "henry_sample_levels": (I, [P, ctypes.POINTER(HenryLevelBatch), I, V]),
        "mlmc_level_stats": (I, [P, I, V, V, I, V, ctypes.POINTER(LevelStats), V]),
        "mlmc_field_stats": (I, [P, I, V, V, I, V, V, V, V, V, V, V]),
        "mlmc_field_exceedance": (I, [P, I, V, I, V, D, V, V]),
        "henry_residual_jacobian": (I, [cfgp, I, I, D, I, V, V, V, V, V, V, V, V, V]),
        "henry_residual_jacobian_noalloc": (I, [cfgp, I, I, D, I, V, V, V, V, V, V, V, V, V]),
        "henry_residual_jacobian_vc": (I, [cfgp, I, I, D, I, V, V, V, V, V, V, V]),
        "henry_fields": (I, [P, I, V, V, I, V, V, V, V]),
        "henry_adjoint": (I, [P, I, V, V, I, I, I, V, V, V, V, V]),
        "henry_level_info": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                 ctypes.POINTER(I)]),
        "henry_launch_count": (ctypes.c_int64, [P]),
        "henry_debug_copy": (I, [P, I, I, I, I, V, ctypes.c_int64]),
        "henry_time_kernel": (I, [P, I, I, I, I, V, ctypes.c_int64, V, ctypes.POINTER(D),
                                  ctypes.POINTER(D), ctypes.POINTER(D)]),
        "henry_probe_fp64": (I, [I, V, ctypes.POINTER(D)]),
        "henry_strerror": (ctypes.c_char_p, [I]),
        "henry_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    """Entry points declared in include/henry.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(\w+)\s*\(", text, re.M)))


def _check(rc: int):
    if rc != 0:
        raise HenryError(rc, load().henry_last_error().decode())


def default_config(**kw) -> HenryConfig:
    cfg = HenryConfig()
    _check(load().henry_default_config(ctypes.byref(cfg)))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _ptr(t, dtype=None, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or NULL for None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class LevelInfo:
    nx: int
    ny: int
    nt: int
    n_mg: int


class Context:
    """A henry_ctx: levels 0..cfg.nlevels-1 and their device workspaces."""

    def __init__(self, cfg: HenryConfig):
        self.lib = load()
        self.cfg = cfg
        h = ctypes.c_void_p()
        _check(self.lib.henry_create_levels(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h:
            self.lib.henry_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_info(self, level: int) -> LevelInfo:
        v = [ctypes.c_int() for _ in range(4)]
        _check(self.lib.henry_level_info(self._h, level, *[ctypes.byref(x) for x in v]))
        return LevelInfo(*[x.value for x in v])

    def field_shape(self, level):
        """Shape of one sample's c / p output at `level`: (ny, nx) cells, or
        (ny + 1, nx) unknown nodes with the vertex-centred variant."""
        li = self.level_info(level)
        return (li.ny + 1, li.nx) if self.cfg.discretisation == DISC_VERTEX else (li.ny, li.nx)

    def debug_copy(self, level, role, mg_level, what, nbytes):
        """henry_debug_copy into a host numpy byte buffer."""
        buf = np.zeros(nbytes, dtype=np.uint8)
        _check(self.lib.henry_debug_copy(self._h, level, role, mg_level, what,
                                         buf.ctypes.data_as(ctypes.c_void_p), nbytes))
        return buf

    def time_kernel(self, level, role, which, reps=20, flush=None, stream=None):
        """henry_time_kernel: (avg ms per launch, algorithmic bytes, flops).
        flush: a CUDA tensor larger than L2, overwritten before every timed
        launch (each launch then starts cold and is timed on its own)."""
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        fb = 0 if flush is None else flush.numel() * flush.element_size()
        _check(self.lib.henry_time_kernel(self._h, level, role, which, reps, _ptr(flush), fb,
                                          _stream(stream), ctypes.byref(ms), ctypes.byref(by),
                                          ctypes.byref(fl)))
        return ms.value, by.value, fl.value

    def launch_count(self) -> int:
        return int(self.lib.henry_launch_count(self._h))

    def solve(self, level, xi, logk=None, want_c=False, want_p=False, want_iters=False,
              stream=None):
        """henry_solve: returns dict(q [B,NQ], status [B], c, p, iters as asked)."""
        import torch
        B = xi.shape[0]
        li = self.level_info(level)
        dev = xi.device
        q = torch.empty((B, NQ), dtype=torch.float64, device=dev)
        st = torch.empty((B,), dtype=torch.int32, device=dev)
        c = torch.empty((B,) + self.field_shape(level), dtype=torch.float64, device=dev) \
            if want_c else None
        p = torch.empty((B,) + self.field_shape(level), dtype=torch.float64, device=dev) \
            if want_p else None
        it = torch.empty((B,), dtype=torch.int32, device=dev) if want_iters else None
        _check(self.lib.henry_solve(
            self._h, level, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"),
            _ptr(logk, torch.float64, (B, li.ny, li.nx), "logk"), B, _ptr(q), _ptr(c), _ptr(p),
            _ptr(st), _ptr(it), _stream(stream)))
        return {"q": q, "status": st, "c": c, "p": p, "iters": it}

    def solve_series(self, level, xi, every, logk=None, stream=None):
        """henry_solve_series: dict(series [B, nt/every, NQ], q [B, NQ], status [B])."""
        import torch
        B = xi.shape[0]
        li = self.level_info(level)
        dev = xi.device
        series = torch.empty((B, li.nt // every, NQ), dtype=torch.float64, device=dev)
        q = torch.empty((B, NQ), dtype=torch.float64, device=dev)
        st = torch.empty((B,), dtype=torch.int32, device=dev)
        _check(self.lib.henry_solve_series(
            self._h, level, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"),
            _ptr(logk, torch.float64, (B, li.ny, li.nx), "logk"), B, int(every), _ptr(series),
            _ptr(q), _ptr(st), _stream(stream)))
        return {"series": series, "q": q, "status": st}

    def sample_pairs(self, level, xi, want_c=False, stream=None):
        """henry_sample_pairs: (q_fine, q_coarse or None, c_fine, c_coarse, status)."""
        import torch
        B = xi.shape[0]
        dev = xi.device
        li = self.level_info(level)
        qf = torch.empty((B, NQ), dtype=torch.float64, device=dev)
        qc = torch.empty((B, NQ), dtype=torch.float64, device=dev) if level > 0 else None
        cf = torch.empty((B,) + self.field_shape(level), dtype=torch.float64, device=dev) \
            if want_c else None
        cc = None
        if want_c and level > 0:
            cc = torch.empty((B,) + self.field_shape(level - 1), dtype=torch.float64, device=dev)
        st = torch.empty((B,), dtype=torch.int32, device=dev)
        _check(self.lib.henry_sample_pairs(
            self._h, level, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"), B, _ptr(qf),
            _ptr(qc), _ptr(cf), _ptr(cc), _ptr(st), _stream(stream)))
        return qf, qc, cf, cc, st

    def set_schedule(self, level, vcycles, nu1, nu2, mg_small_cells=512, jac_lag=0, res_rows=0,
                     mg_tb_cells=0, jac_keep=0, **_):
        """henry_set_schedule: the multigrid schedule of one MLMC level."""
        sc = HenrySchedule(vcycles, nu1, nu2, mg_small_cells, jac_lag, res_rows, mg_tb_cells,
                           jac_keep)
        _check(self.lib.henry_set_schedule(self._h, level, ctypes.byref(sc)))

    def sample_levels(self, xis, want_c=False, stream=None):
        """henry_sample_levels: the pairs of several levels at once, one graph
        launch per coarse time step. xis: {level: xi [B, n_xi]}. Returns
        {level: (q_fine, q_coarse or None, c_fine, c_coarse, status)}."""
        import torch
        arr = (HenryLevelBatch * len(xis))()
        out, keep = {}, []
        for i, (level, xi) in enumerate(sorted(xis.items())):
            B = xi.shape[0]
            dev = xi.device
            li = self.level_info(level)
            qf = torch.empty((B, NQ), dtype=torch.float64, device=dev)
            qc = torch.empty((B, NQ), dtype=torch.float64, device=dev) if level > 0 else None
            cf = torch.empty((B,) + self.field_shape(level), dtype=torch.float64, device=dev) \
                if want_c else None
            cc = None
            if want_c and level > 0:
                cc = torch.empty((B,) + self.field_shape(level - 1), dtype=torch.float64,
                                 device=dev)
            st = torch.empty((B,), dtype=torch.int32, device=dev)
            p = lambda t, name=None, **kw: _ptr(t, **kw)
            arr[i] = HenryLevelBatch(level, B, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"),
                                     p(qf), p(qc), p(cf), p(cc), p(st))
            out[level] = (qf, qc, cf, cc, st)
            keep.append(xi)
        _check(self.lib.henry_sample_levels(self._h, arr, len(xis), _stream(stream)))
        return out

    def level_stats(self, level, q_fine, q_coarse, status, stats: LevelStats, stream=None):
        """mlmc_level_stats (synchronous): merges the batch into `stats`."""
        import torch
        B = q_fine.shape[0]
        _check(self.lib.mlmc_level_stats(
            self._h, level, _ptr(q_fine, torch.float64, (B, NQ), "q_fine"),
            _ptr(q_coarse, torch.float64, (B, NQ), "q_coarse"), B,
            _ptr(status, torch.int32, (B,), "status"), ctypes.byref(stats), _stream(stream)))
        return stats

    def field_stats(self, level, c_fine, c_coarse, status, acc: dict, stream=None):
        """mlmc_field_stats: acc holds device tensors n, mean_f, m2_f, mean_d, m2_d."""
        import torch
        B = c_fine.shape[0]
        _check(self.lib.mlmc_field_stats(
            self._h, level, _ptr(c_fine, torch.float64, None, "c_fine"),
            _ptr(c_coarse, torch.float64, None, "c_coarse"), B,
            _ptr(status, torch.int32, (B,), "status"), _ptr(acc["n"], torch.int64),
            _ptr(acc["mean_f"], torch.float64), _ptr(acc["m2_f"], torch.float64),
            _ptr(acc["mean_d"], torch.float64), _ptr(acc["m2_d"], torch.float64),
            _stream(stream)))
        return acc

    def field_exceedance(self, level, c, status, threshold, count, stream=None):
        """mlmc_field_exceedance: count (device int64 [ny*nx]) += samples with
        c > threshold, per cell."""
        import torch
        B = c.shape[0]
        _check(self.lib.mlmc_field_exceedance(
            self._h, level, _ptr(c, torch.float64, None, "c"), B,
            _ptr(status, torch.int32, (B,), "status"), float(threshold),
            _ptr(count, torch.int64), _stream(stream)))
        return count

    def adjoint(self, level, xi, logk=None, qoi="Q_S", ckpt_every=8, want_logk=True, stream=None):
        """henry_adjoint: (q [B], dq_dxi [B,n_xi], dq_dlogk [B,ny,nx] or None, status [B])."""
        import torch
        B = xi.shape[0]
        li = self.level_info(level)
        dev = xi.device
        qid = {"Q_S": 0, "toe": 2}[qoi]
        q = torch.empty((B,), dtype=torch.float64, device=dev)
        g = torch.empty((B, self.cfg.n_xi), dtype=torch.float64, device=dev)
        gl = torch.empty((B, li.ny, li.nx), dtype=torch.float64, device=dev) if want_logk else None
        st = torch.empty((B,), dtype=torch.int32, device=dev)
        _check(self.lib.henry_adjoint(
            self._h, level, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"),
            _ptr(logk, torch.float64, (B, li.ny, li.nx), "logk"), B, qid, ckpt_every, _ptr(q),
            _ptr(g), _ptr(gl), _ptr(st), _stream(stream)))
        return q, g, gl, st

    def fields(self, level, xi, logk=None, stream=None):
        import torch
        B = xi.shape[0]
        li = self.level_info(level)
        dev = xi.device
        phi = torch.empty((B, li.ny, li.nx), dtype=torch.float64, device=dev)
        K = torch.empty_like(phi)
        qin = torch.empty((B, li.ny), dtype=torch.float64, device=dev)
        _check(self.lib.henry_fields(self._h, level, _ptr(xi, torch.float64, (B, self.cfg.n_xi), "xi"),
                                     _ptr(logk, torch.float64, (B, li.ny, li.nx), "logk"), B,
                                     _ptr(phi), _ptr(K), _ptr(qin), _stream(stream)))
        return phi, K, qin


def probe_fp64(reps=40, stream=None):
    """henry_probe_fp64: measured FP64 FMA throughput of the GPU [TFLOP/s]."""
    v = ctypes.c_double()
    _check(load().henry_probe_fp64(int(reps), _stream(stream), ctypes.byref(v)))
    return v.value


def new_field_accumulator(ny, nx, device="cuda"):
    import torch
    z = lambda: torch.zeros((ny, nx), dtype=torch.float64, device=device)
    return {"n": torch.zeros((ny, nx), dtype=torch.int64, device=device), "mean_f": z(),
            "m2_f": z(), "mean_d": z(), "m2_d": z()}


def residual_jacobian(cfg: HenryConfig, tau, phi, K, qin, p, c, c_old, want_J=True, stream=None,
                      noalloc=False):
    """henry_residual_jacobian (or, with noalloc=True, the entry point that
    allocates no device memory): R [B,2,ny,nx] and J [B,20,ny,nx] (or None)."""
    import torch
    B, ny, nx = p.shape
    R = torch.empty((B, 2, ny, nx), dtype=torch.float64, device=p.device)
    J = torch.empty((B, 20, ny, nx), dtype=torch.float64, device=p.device) if want_J else None
    f64 = torch.float64
    fn = load().henry_residual_jacobian_noalloc if noalloc else load().henry_residual_jacobian
    _check(fn(
        ctypes.byref(cfg), nx, ny, float(tau), B, _ptr(phi, f64, (B, ny, nx), "phi"),
        _ptr(K, f64, (B, ny, nx), "K"), _ptr(qin, f64, (B, ny), "qin"), _ptr(p, f64, None, "p"),
        _ptr(c, f64, (B, ny, nx), "c"), _ptr(c_old, f64, (B, ny, nx), "c_old"), _ptr(R), _ptr(J),
        _stream(stream)))
    return R, J


def residual_jacobian_vc(cfg: HenryConfig, tau, xi, p, c, c_old, want_J=True, stream=None):
    """henry_residual_jacobian_vc: R [B,2,ny+1,nx] and J [B,20,ny+1,nx] (or
    None) of the vertex-centred variant; p, c, c_old [B, ny+1, nx] at the
    unknown nodes (nx, ny: cells of the grid)."""
    import torch
    B, ny1, nx = p.shape
    R = torch.empty((B, 2, ny1, nx), dtype=torch.float64, device=p.device)
    J = torch.empty((B, 20, ny1, nx), dtype=torch.float64, device=p.device) if want_J else None
    f64 = torch.float64
    _check(load().henry_residual_jacobian_vc(
        ctypes.byref(cfg), nx, ny1 - 1, float(tau), B, _ptr(xi, f64, (B, cfg.n_xi), "xi"),
        _ptr(p, f64, (B, ny1, nx), "p"), _ptr(c, f64, (B, ny1, nx), "c"),
        _ptr(c_old, f64, (B, ny1, nx), "c_old"), _ptr(R), _ptr(J), _stream(stream)))
    return R, J


def henry_qoi(ctx: Context, level: int, xi, logk=None, qoi="Q_S", ckpt_every=8):
    """Differentiable QoI of a batch of Henry solves: returns q [B]; its
    gradient with respect to xi (and logk, if given) comes from the discrete
    adjoint (henry_adjoint), computed together with q in the forward call."""
    import torch

    class _HenryQoI(torch.autograd.Function):
        @staticmethod
        def forward(fctx, xi_, logk_):
            q, g, gl, st = ctx.adjoint(level, xi_.detach().contiguous(),
                                       None if logk_ is None else logk_.detach().contiguous(),
                                       qoi=qoi, ckpt_every=ckpt_every, want_logk=logk_ is not None)
            fctx.save_for_backward(g, gl if gl is not None else torch.empty(0, device=xi_.device))
            fctx.has_logk = logk_ is not None
            fctx.status = st
            return q

        @staticmethod
        def backward(fctx, grad_q):
            g, gl = fctx.saved_tensors
            gx = grad_q[:, None] * g
            glk = grad_q[:, None, None] * gl if fctx.has_logk else None
            return gx, glk

    return _HenryQoI.apply(xi, logk)
