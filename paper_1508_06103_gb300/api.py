"""Python binding of the C ABI with torch tensors for device memory and streams.

Each wrapper only marshals arguments (pointers, sizes, the current CUDA
stream) and calls the library; the arithmetic runs in the CUDA kernels.
Vectors are 1-D torch tensors on the current CUDA device in the paper's
point-block order U[((n*N + j)*3 + c)] (c = C, G, f).
"""

from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check


def _stream(stream: Optional[torch.cuda.Stream] = None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor], dtype=torch.float64) -> C.c_void_p:
    if t is None:
        return C.c_void_p(None)
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    return C.c_void_p(t.data_ptr())


class Problem:
    """Handle of one discrete KKT system F_h (kkt_create)."""

    def __init__(self, cells: Sequence[int], lengths: Sequence[float], nt: int, dt: float,
                 a_cell: np.ndarray, v_cell: np.ndarray, sensor_node: np.ndarray, beta1: float, beta2: float,
                 theta: float = 0.5, dirichlet_faces: int = 1):
        self._lib = _lib.load()
        g = _lib.KktGrid(int(cells[0]), int(cells[1]), int(cells[2]), float(lengths[0]), float(lengths[1]),
                         float(lengths[2]), int(dirichlet_faces))
        a = np.ascontiguousarray(a_cell, dtype=np.float64)
        v = np.ascontiguousarray(v_cell, dtype=np.float64).reshape(-1)
        s = np.ascontiguousarray(sensor_node, dtype=np.int32)
        h = C.c_void_p()
        check(self._lib.kkt_create(C.byref(g), int(nt), float(dt), a.ctypes.data_as(C.c_void_p),
                                   v.ctypes.data_as(C.c_void_p),
                                   s.ctypes.data_as(C.c_void_p) if s.size else None, int(s.size),
                                   float(beta1), float(beta2), float(theta), C.byref(h)), "kkt_create")
        self.h = h
        nx, ny, nz, lv = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        n = C.c_longlong()
        check(self._lib.kkt_sizes(h, C.byref(nx), C.byref(ny), C.byref(nz), C.byref(lv), C.byref(n)), "kkt_sizes")
        self.nodes = (nx.value, ny.value, nz.value)
        self.N = nx.value * ny.value * nz.value
        self.levels = lv.value
        self.n = n.value
        self.nsens = int(s.size)

    @classmethod
    def from_workload(cls, w, cells=None, M=None) -> "Problem":
        p = cls(w.cells, w.lengths, w.M, w.tau, w.a_cell, w.v_cell, w.sensor_nodes(), w.beta1, w.beta2,
                w.theta, w.dirichlet_faces)
        if getattr(w, "reg", "h1h1") != "h1h1":
            p.set_regularization(w.reg)
        if getattr(w, "element", "q1") != "q1":
            p.set_element(w.element)
        return p

    def set_regularization(self, reg: str) -> None:
        """'h1h1' (N_beta, Eq. 3) or 'h1l2' (Sec. 4, Example 2); before building preconditioners."""
        check(self._lib.kkt_set_regularization(self.h, {"h1h1": 0, "h1l2": 1}[reg]), "kkt_set_regularization")

    def set_element(self, element: str) -> None:
        """'q1' (trilinear hexahedra) or 'p1' (Kuhn split into tetrahedra); before building preconditioners."""
        check(self._lib.kkt_set_element(self.h, {"q1": 0, "p1": 1}[element]), "kkt_set_element")

    def close(self):
        if self.h is not None and self.h.value:
            self._lib.kkt_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- vectors -------------------------------------------------------------
    def zeros(self, dtype=torch.float64) -> torch.Tensor:
        return torch.zeros(self.n, dtype=dtype, device="cuda")

    def rhs(self, c_obs: torch.Tensor, c0: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
            stream=None) -> torch.Tensor:
        b = out if out is not None else self.zeros()
        check(self._lib.kkt_rhs(self.h, _ptr(c_obs.contiguous()) if self.nsens else None, _ptr(c0), _ptr(b),
                                _stream(stream)), "kkt_rhs")
        return b

    def apply(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        prec = 64 if x.dtype == torch.float64 else 32
        y = out if out is not None else torch.empty_like(x)
        check(self._lib.kkt_apply(self.h, _ptr(x, x.dtype), _ptr(y, x.dtype), prec, _stream(stream)), "kkt_apply")
        return y

    def residual(self, b: torch.Tensor, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
        r = out if out is not None else torch.empty_like(b)
        check(self._lib.kkt_residual(self.h, _ptr(b), _ptr(x), _ptr(r), _stream(stream)), "kkt_residual")
        return r

    def recover_source(self, U: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        f = out if out is not None else torch.empty(self.levels * self.N, dtype=torch.float64, device="cuda")
        check(self._lib.recover_source(self.h, _ptr(U), _ptr(f), _stream(stream)), "recover_source")
        return f.view(self.levels, self.N)


class RAS:
    """One-level space-time RAS with ILU(0) subdomain solves (ras_setup)."""

    def __init__(self, prob: Problem, nsub: Sequence[int], overlap: int, factor_prec: int = 64, local: str = "ilu0",
                 shape: Optional[Sequence[int]] = None):
        """factor_prec 64, 32 or 16 (BF16 storage); local "ilu0", "lu" (exact, FP64 only), "ilu1" (ILU(1))
        or "bilu0" (3x3 point-block ILU(0)); the last two in FP64 or FP32.

        shape: None (chosen by the library) or (chunk points, ring buffers, lanes, placement) for
        ras_setup_shape, placement 1 = local vectors in shared memory, 2 = in global memory, 0 = any.
        """
        self._lib = _lib.load()
        self.prob = prob
        ns = (C.c_int * 4)(*[int(v) for v in nsub])
        h = C.c_void_p()
        loc = {"ilu0": 0, "lu": 1, "ilu1": 2, "bilu0": 3}[local]
        if shape is None:
            check(self._lib.ras_setup(prob.h, ns, int(overlap), loc, int(factor_prec), C.byref(h)), "ras_setup")
        else:
            sh = (C.c_int * 4)(*[int(v) for v in shape])
            check(self._lib.ras_setup_shape(prob.h, ns, int(overlap), loc, int(factor_prec), sh, C.byref(h)),
                  "ras_setup_shape")
        self.h = h

    def apply(self, r: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        z = out if out is not None else torch.empty_like(r)
        check(self._lib.ras_apply(self.h, _ptr(r), _ptr(z), _stream(stream)), "ras_apply")
        return z

    def refactor(self, stream=None) -> None:
        check(self._lib.ras_refactor(self.h, _stream(stream)), "ras_refactor")

    def apply_static(self, r: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """ras_apply with the library's fixed scratch array (allocates nothing)."""
        z = out if out is not None else torch.empty_like(r)
        check(self._lib.ras_apply_static(self.h, _ptr(r), _ptr(z), _stream(stream)), "ras_apply_static")
        return z

    def info(self):
        """dict(nbox, points, factor_values, value_bytes)."""
        nb, pts, fv, vb = C.c_int(), C.c_longlong(), C.c_longlong(), C.c_int()
        check(self._lib.ras_info(self.h, C.byref(nb), C.byref(pts), C.byref(fv), C.byref(vb)), "ras_info")
        return dict(nbox=nb.value, points=pts.value, factor_values=fv.value, value_bytes=vb.value)

    def solve_shape(self):
        """dict(chunk_points, stages, lanes, smem_vectors) of the subdomain solve."""
        ch, ns, ln, sv = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(self._lib.ras_solve_shape(self.h, C.byref(ch), C.byref(ns), C.byref(ln), C.byref(sv)),
              "ras_solve_shape")
        return dict(chunk_points=ch.value, stages=ns.value, lanes=ln.value, smem_vectors=bool(sv.value))

    def status(self, stream=None) -> int:
        """The device status word (ras_status); raises KktError for 1 (zero pivot) and 2 (copy wait gave up)."""
        code = C.c_int()
        check(self._lib.ras_status(self.h, C.byref(code), _stream(stream)), "ras_status")
        return code.value

    def selftest_wait(self, limit_ms: float, stream=None) -> None:
        """Run the bounded-wait self-test kernel (ras_selftest_wait)."""
        check(self._lib.ras_selftest_wait(self.h, float(limit_ms), _stream(stream)), "ras_selftest_wait")

    def timing(self, kernel: int = 0):
        """(total ms, launches) since the last reset: kernel 0 subdomain solve, 1 factorisation."""
        ms, n = C.c_double(), C.c_longlong()
        check(self._lib.ras_timing_read(self.h, int(kernel), C.byref(ms), C.byref(n)), "ras_timing_read")
        return ms.value, n.value

    def close(self):
        if self.h is not None and self.h.value:
            self._lib.ras_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Coarse:
    """Coarse space-time level of the two-level method (coarse_setup)."""

    def __init__(self, prob: Problem, ccells: Sequence[int], cnt: int, nsub_c: Sequence[int], c_overlap: int = 1,
                 c_rtol: float = 0.1, c_maxit: int = 4, factor_prec: int = 64):
        self._lib = _lib.load()
        self.prob = prob
        ns = (C.c_int * 4)(*[int(v) for v in nsub_c])
        h = C.c_void_p()
        check(self._lib.coarse_setup(prob.h, int(ccells[0]), int(ccells[1]), int(ccells[2]), int(cnt), ns,
                                     int(c_overlap), float(c_rtol), int(c_maxit), int(factor_prec), C.byref(h)),
              "coarse_setup")
        self.h = h

    def apply(self, fine: RAS, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        z = out if out is not None else torch.empty_like(x)
        check(self._lib.two_level_apply(self.h, fine.h, _ptr(x), _ptr(z), _stream(stream)), "two_level_apply")
        return z

    def refactor(self, stream=None) -> None:
        check(self._lib.coarse_refactor(self.h, _stream(stream)), "coarse_refactor")

    def refactor_with(self, fine: RAS, stream=None) -> None:
        """Refactor `fine` and this coarse level together (two_level_refactor)."""
        check(self._lib.two_level_refactor(self.h, fine.h, _stream(stream)), "two_level_refactor")

    def close(self):
        if self.h is not None and self.h.value:
            self._lib.coarse_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(_lib.load().kkt_launch_count())


def fma_peak(precision: int = 64, stream=None):
    """(TFLOP/s, ms) of the device's multiply-add rate in FP64 or FP32 (kkt_fma_peak)."""
    tf, ms = C.c_double(), C.c_double()
    check(_lib.load().kkt_fma_peak(int(precision), C.byref(tf), C.byref(ms), _stream(stream)), "kkt_fma_peak")
    return tf.value, ms.value


def mma_peak(stream=None):
    """(TFLOP/s, ms) of the device's FP64 tensor-core (MMA) rate (kkt_mma_peak)."""
    tf, ms = C.c_double(), C.c_double()
    check(_lib.load().kkt_mma_peak(C.byref(tf), C.byref(ms), _stream(stream)), "kkt_mma_peak")
    return tf.value, ms.value


def timing_enable(on: bool) -> bool:
    return bool(_lib.load().kkt_timing_enable(int(on)))


def matvec_timing(prob: Problem):
    """(total ms, launches) of the solver's FP64 matvecs on prob since the last reset."""
    ms, n = C.c_double(), C.c_longlong()
    check(_lib.load().kkt_timing_read(prob.h, C.byref(ms), C.byref(n)), "kkt_timing_read")
    return ms.value, n.value


def timing_reset(prob: Optional[Problem] = None, ras: Optional["RAS"] = None) -> None:
    _lib.load().kkt_timing_reset(prob.h if prob else None, ras.h if ras else None)


def gmres_solve(prob: Problem, b: torch.Tensor, x: Optional[torch.Tensor] = None, ras: Optional[RAS] = None,
                coarse: Optional[Coarse] = None, restart: int = 30, rtol: float = 1e-8, maxit: int = 1000,
                flexible: Optional[bool] = None, stream=None):
    """Solve F_h x = b; returns (x, status, iterations, true relative residual)."""
    lib = _lib.load()
    if x is None:
        x = torch.zeros_like(b)
    flex = (coarse is not None) if flexible is None else bool(flexible)
    it = C.c_int()
    rel = C.c_double()
    st = lib.gmres_solve(prob.h, ras.h if ras else None, coarse.h if coarse else None, _ptr(b), _ptr(x),
                         int(restart), float(rtol), int(maxit), int(flex), C.byref(it), C.byref(rel), _stream(stream))
    check(st, "gmres_solve")
    return x, st, it.value, rel.value


def local_pattern(local: str):
    """Slots per row type (C, G, f) of an interior point under a local solver (ras_local_pattern)."""
    counts = (C.c_int * 3)()
    check(_lib.load().ras_local_pattern({"ilu0": 0, "ilu1": 2, "bilu0": 3}[local], counts), "ras_local_pattern")
    return list(counts)


def reduced_solve(prob: Problem, c_obs: torch.Tensor, c0: Optional[torch.Tensor] = None, restart: int = 30,
                  rtol: float = 1e-10, maxit: int = 2000, step_rtol: float = 1e-13, stream=None):
    """KKT solution by the reduced-space method (reduced_solve); returns
    (U, status, outer iterations, reduced relative residual, stats dict)."""
    lib = _lib.load()
    U = prob.zeros()
    it = C.c_int()
    rel = C.c_double()
    stats = (C.c_longlong * 4)()
    st = lib.reduced_solve(prob.h, _ptr(c_obs) if prob.nsens else None, _ptr(c0) if c0 is not None else None,
                           _ptr(U), int(restart), float(rtol), int(maxit), float(step_rtol), C.byref(it),
                           C.byref(rel), stats, _stream(stream))
    check(st, "reduced_solve")
    names = ("hess_applies", "step_solves", "step_iterations", "step_iterations_max")
    return U, st, it.value, rel.value, dict(zip(names, list(stats)))


def checkpoint_save(path: str, x: torch.Tensor, **meta) -> None:
    """Write the iterate x of a solve (any device) and scalar metadata (iterations, residual,
    ...) to an .npz file.  A restarted (F)GMRES starts every cycle from a fresh Krylov space, so
    the iterate is the whole state: resuming is gmres_solve(prob, b, x=checkpoint_load(...)[0])."""
    arrays = {"x": x.detach().cpu().numpy()}
    for k, v in meta.items():
        arrays["meta_" + k] = np.asarray(v)
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def checkpoint_load(path: str, device: str = "cuda"):
    """(x on `device`, metadata dict) from checkpoint_save."""
    with np.load(path) as z:
        x = torch.from_numpy(z["x"].copy()).to(device)
        meta = {k[5:]: z[k].item() if z[k].ndim == 0 else z[k] for k in z.files if k.startswith("meta_")}
    return x, meta


def _handles(probs: Sequence[Problem]):
    return (C.c_void_p * len(probs))(*[p.h.value for p in probs])


class BatchRAS(RAS):
    """One-level RAS of several independent problems in one set of launches (ras_setup_batch).

    Vectors concatenate the problems' unknowns in the order of `probs`.
    """

    def __init__(self, probs: Sequence[Problem], nsub: Sequence[int], overlap: int, factor_prec: int = 32,
                 shape: Optional[Sequence[int]] = None):
        self._lib = _lib.load()
        self.prob = probs[0]
        self.probs = list(probs)
        self.offsets = np.cumsum([0] + [p.n for p in probs]).tolist()
        ns = (C.c_int * 4)(*[int(v) for v in nsub])
        sh = None if shape is None else (C.c_int * 4)(*[int(v) for v in shape])
        h = C.c_void_p()
        check(self._lib.ras_setup_batch(_handles(probs), len(probs), ns, int(overlap), int(factor_prec), sh,
                                        C.byref(h)), "ras_setup_batch")
        self.h = h

    @property
    def n(self) -> int:
        return int(self.offsets[-1])


def autotune(probs: Sequence[Problem], nsub: Sequence[int], overlap: int, factor_prec: int = 32, reps: int = 3,
             cache_path: Optional[str] = None):
    """(shape, ms per apply) of the fastest subdomain-solve shape on these problems (ras_autotune)."""
    ns = (C.c_int * 4)(*[int(v) for v in nsub])
    out = (C.c_int * 4)()
    ms = C.c_double()
    check(_lib.load().ras_autotune(_handles(probs), len(probs), ns, int(overlap), int(factor_prec), int(reps),
                                   cache_path.encode() if cache_path else None, out, C.byref(ms)), "ras_autotune")
    return tuple(out), ms.value


def gmres_solve_batch(probs: Sequence[Problem], ras: BatchRAS, b: torch.Tensor, x: Optional[torch.Tensor] = None,
                      restart: int = 30, rtol: float = 1e-8, maxit: int = 1000, stream=None):
    """Solve every problem's F_k x_k = b_k together; returns (x, status, per-problem lists of
    status, iterations and true relative residuals)."""
    lib = _lib.load()
    if x is None:
        x = torch.zeros_like(b)
    n = len(probs)
    its, rel, sts = (C.c_int * n)(), (C.c_double * n)(), (C.c_int * n)()
    st = lib.gmres_solve_batch(_handles(probs), n, ras.h, _ptr(b), _ptr(x), int(restart), float(rtol), int(maxit),
                               its, rel, sts, _stream(stream))
    check(st, "gmres_solve_batch")
    return x, st, list(sts), list(its), list(rel)
