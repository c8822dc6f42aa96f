"""Python face of the C ABI: the same entry-point names as include/spsvm.h,
taking torch tensors for device memory and the current torch CUDA stream.
Only argument marshalling happens here."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import (SPSVM_BF16SPLIT, SPSVM_FP32, check, ptr, stream_ptr,  # noqa: F401
                   spsvm_kmat, spsvm_options, spsvm_points, spsvm_problem, spsvm_step)


def _lib():
    return L.load()


def _prec(p):
    if isinstance(p, str):
        return L.PRECISIONS[p]
    return int(p)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")


# ---------------------------------------------------------------- points
@dataclass
class Points:
    """Prepared points (spsvm_points) with the buffers that back it."""
    X: torch.Tensor
    norms: torch.Tensor
    hi: torch.Tensor | None
    lo: torch.Tensor | None
    ldh: int
    mid: torch.Tensor | None = None

    def struct(self):
        s = spsvm_points()
        s.X = ptr(self.X)
        s.n, s.d = self.X.shape
        s.ldx = self.X.stride(0)
        s.norms = ptr(self.norms)
        s.hi = ptr(self.hi)
        s.lo = ptr(self.lo)
        s.ldh = self.ldh
        s.mid = ptr(self.mid)
        return s


def spsvm_prepare_points(X: torch.Tensor, precision="fp32") -> Points:
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.stride(1) == 1
    n, d = X.shape
    ldh = ((d + 63) // 64) * 64
    p = _prec(precision)
    norms = torch.empty(n, dtype=torch.float32, device=X.device)
    hi = mid = lo = None
    if p == SPSVM_BF16SPLIT:
        hi = torch.empty((n, ldh), dtype=torch.bfloat16, device=X.device)
        mid = torch.empty((n, ldh), dtype=torch.bfloat16, device=X.device)
        lo = torch.empty((n, ldh), dtype=torch.bfloat16, device=X.device)
    P = Points(X, norms, hi, lo, ldh, mid)
    s = P.struct()
    check(_lib().spsvm_prepare_points(C.byref(s), p, stream_ptr()), "spsvm_prepare_points")
    return P


# ---------------------------------------------------------------- K storage
@dataclass
class KMat:
    """A stored kernel matrix (spsvm_kmat) backed by a torch tensor."""
    buf: torch.Tensor
    format: int
    n: int
    rows: int
    ld: int
    plane: int

    def struct(self, rows=None):
        s = spsvm_kmat()
        s.data = ptr(self.buf)
        s.format = self.format
        s.n = self.n
        s.rows = self.rows if rows is None else rows
        s.ld = self.ld
        s.plane = self.plane
        return s

    def to_float(self, rows=None):
        """FP32 copy of rows x n (hi + lo for BF16SPLIT), on the device."""
        r = self.rows if rows is None else rows
        if self.format == SPSVM_FP32:
            return self.buf.view(-1)[: r * self.ld].view(r, self.ld)[:, : self.n].clone()
        flat = self.buf.view(-1)
        hi = flat[: r * self.ld].view(r, self.ld)[:, : self.n].float()
        lo = flat[self.plane: self.plane + r * self.ld].view(r, self.ld)[:, : self.n].float()
        return hi + lo


def kmat_empty(n, rows, precision="fp32", device="cuda", ld=None):
    p = _prec(precision)
    ld = ld if ld is not None else ((n + 127) // 128) * 128
    if p == SPSVM_FP32:
        buf = torch.zeros(max(1, rows * ld), dtype=torch.float32, device=device)
        return KMat(buf, p, n, rows, ld, 0)
    plane = rows * ld
    buf = torch.zeros(max(1, 2 * plane), dtype=torch.bfloat16, device=device)
    return KMat(buf, p, n, rows, ld, plane)


def spsvm_kernel_block(P: Points, idx: torch.Tensor, gamma, precision, out: KMat, row0=0,
                       scratch=None):
    s = P.struct()
    k = out.struct()
    m = int(idx.numel())
    sb = _lib().spsvm_kernel_block_scratch_bytes(m, P.X.shape[1], _prec(precision))
    if scratch is None:
        scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=P.X.device)
    check(_lib().spsvm_kernel_block(C.byref(s), ptr(idx), m, float(gamma), _prec(precision),
                                    C.byref(k), int(row0), ptr(scratch), scratch.numel(),
                                    stream_ptr()),
          "spsvm_kernel_block")
    return out


def spsvm_score_candidates(P: Points, y, o, idx, gamma, lam, precision):
    n = P.X.shape[0]
    kappa = int(idx.numel())
    dev = P.X.device
    g = torch.empty(kappa, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    delta = torch.empty_like(g)
    sb = _lib().spsvm_score_scratch_bytes(n, P.X.shape[1], kappa)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=dev)
    s = P.struct()
    check(_lib().spsvm_score_candidates(C.byref(s), ptr(y), ptr(o), ptr(idx), kappa, float(gamma),
                                        float(lam), _prec(precision), ptr(g), ptr(h), ptr(delta),
                                        ptr(scratch), sb, stream_ptr()),
          "spsvm_score_candidates")
    return g, h, delta


def spsvm_score_candidates_exact(P: Points, y, o, idx, gamma, lam, precision, bias=None):
    """Exact one-dimensional selection scores: (delta, t), FP64 device
    tensors of the candidates' exact decrease of f and signed minimiser."""
    n, d = P.X.shape
    kappa = int(idx.numel())
    dev = P.X.device
    delta = torch.empty(max(1, kappa), dtype=torch.float64, device=dev)
    t = torch.empty_like(delta)
    sb = _lib().spsvm_score_exact_scratch_bytes(n, d, kappa, _prec(precision))
    scratch = torch.empty(max(256, sb), dtype=torch.uint8, device=dev)
    s = P.struct()
    bb = torch.tensor([float(bias)], dtype=torch.float64, device=dev) if bias is not None else None
    check(_lib().spsvm_score_candidates_exact(C.byref(s), ptr(y), ptr(o), ptr(idx), kappa,
                                              float(gamma), float(lam), _prec(precision), ptr(bb),
                                              ptr(delta), ptr(t), ptr(scratch), sb, stream_ptr()),
          "spsvm_score_candidates_exact")
    return delta[:kappa], t[:kappa]


def spsvm_score_candidates_noalloc(P: Points, y, o, idx, gamma, lam, precision):
    """spsvm_score_candidates without caller scratch: the partial sums go to
    the library's fixed device array (see include/spsvm.h)."""
    kappa = int(idx.numel())
    dev = P.X.device
    g = torch.empty(kappa, dtype=torch.float64, device=dev)
    h = torch.empty_like(g)
    delta = torch.empty_like(g)
    s = P.struct()
    check(_lib().spsvm_score_candidates_noalloc(C.byref(s), ptr(y), ptr(o), ptr(idx), kappa,
                                                float(gamma), float(lam), _prec(precision),
                                                ptr(g), ptr(h), ptr(delta), stream_ptr()),
          "spsvm_score_candidates_noalloc")
    return g, h, delta


def spsvm_outputs(K: KMat, beta, y, o, rows=None):
    n = K.n
    dev = y.device
    active = torch.empty(n, dtype=torch.uint8, device=dev)
    stats = torch.empty(3, dtype=torch.float64, device=dev)
    sb = _lib().spsvm_reduce_scratch_bytes(n)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=dev)
    k = K.struct(rows)
    check(_lib().spsvm_outputs(C.byref(k), ptr(beta), ptr(y), ptr(o), ptr(active), ptr(stats),
                               ptr(scratch), sb, stream_ptr()), "spsvm_outputs")
    return active, stats


def spsvm_gemv(K: KMat, v, u, accumulate=False, rows=None):
    k = K.struct(rows)
    check(_lib().spsvm_gemv(C.byref(k), ptr(v), ptr(u), int(bool(accumulate)), stream_ptr()),
          "spsvm_gemv")
    return u


def spsvm_compact_active(K: KMat, active, w1=None, w2=None, Kc: KMat | None = None, rows=None):
    n = K.n
    r = K.rows if rows is None else rows
    dev = active.device
    w1o = torch.empty(max(1, r), dtype=torch.float64, device=dev) if w1 is not None else None
    w2o = torch.empty(max(1, r), dtype=torch.float64, device=dev) if w2 is not None else None
    nact = torch.zeros(1, dtype=torch.int64, device=dev)
    pos = torch.empty(max(1, n), dtype=torch.int32, device=dev)
    sb = _lib().spsvm_compact_scratch_bytes(n, r)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=dev)
    k = K.struct(rows)
    kc = Kc.struct(rows) if Kc is not None else None
    check(_lib().spsvm_compact_active(C.byref(k), ptr(active), ptr(w1), ptr(w2), ptr(w1o), ptr(w2o),
                                      C.byref(kc) if kc is not None else None, ptr(nact), ptr(pos),
                                      ptr(scratch), sb, stream_ptr()), "spsvm_compact_active")
    return w1o, w2o, nact, pos


def spsvm_gram(Kc: KMat, nact, ns_max, K: KMat, J, lam, precision, rows=None):
    m = K.rows if rows is None else rows
    dev = J.device
    H = torch.empty((max(1, m), max(1, m)), dtype=torch.float64, device=dev)
    sb = _lib().spsvm_gram_scratch_bytes(m, ns_max)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=dev)
    kc = Kc.struct(rows)
    k = K.struct(rows)
    check(_lib().spsvm_gram(C.byref(kc), ptr(nact), int(ns_max), C.byref(k), ptr(J), float(lam),
                            _prec(precision), ptr(H), H.stride(0), ptr(scratch), sb, stream_ptr()),
          "spsvm_gram")
    return H[:m, :m]


def spsvm_cholesky(H: torch.Tensor, tensor_cores=True):
    """In-place lower Cholesky factor of H (FP64, square); returns info.
    tensor_cores selects the FP64-faithful tensor-core trailing update."""
    m = H.shape[0]
    info = torch.zeros(1, dtype=torch.int32, device=H.device)
    wb = _lib().spsvm_cholesky_work_bytes(m) if tensor_cores else 0
    work = torch.empty(max(1, wb), dtype=torch.uint8, device=H.device) if wb else None
    check(_lib().spsvm_cholesky(ptr(H), m, H.stride(0), ptr(info), ptr(work), wb, stream_ptr()),
          "spsvm_cholesky")
    return int(info.item())


def spsvm_solve_mixed(H: torch.Tensor, b: torch.Tensor, shift=0.0, max_iter=30, tol=1e-13):
    """Solves (H + shift I) x = b (H FP64, full symmetric, not overwritten) with
    an FP32 factor and FP64 refinement.  Returns (info, status, x, iters,
    backward_error): info != 0 when the FP32 factorisation broke down."""
    m = H.shape[0]
    wb = _lib().spsvm_mixed_work_bytes(m)
    work = torch.empty(max(256, wb), dtype=torch.uint8, device=H.device)
    info = torch.zeros(1, dtype=torch.int32, device=H.device)
    check(_lib().spsvm_cholesky_mixed(ptr(H), m, H.stride(0), float(shift), ptr(info), ptr(work),
                                      wb, stream_ptr()), "spsvm_cholesky_mixed")
    inf = int(info.item())
    x = torch.zeros(m, dtype=torch.float64, device=H.device)
    if inf != 0:
        return inf, None, x, 0, None
    it = C.c_int32()
    be = C.c_double()
    st = _lib().spsvm_solve_mixed(ptr(H), m, H.stride(0), float(shift), ptr(b), ptr(x),
                                  int(max_iter), float(tol), C.byref(it), C.byref(be), ptr(work),
                                  wb, stream_ptr())
    if st not in (L.SPSVM_OK, L.SPSVM_ERR_NO_CONVERGE):
        check(st, "spsvm_solve_mixed")
    return 0, st, x, it.value, be.value


def spsvm_solve_lowrank(Ha: torch.Tensor, H: torch.Tensor, Wt: torch.Tensor, sign: torch.Tensor,
                        b: torch.Tensor, max_iter=30, tol=1e-13, extra_rhs=()):
    """Solves H x = b where H = Ha + W^T diag(sign) W (all FP64 full
    symmetric on the device; Wt = W^T, m x k FP32; sign FP32 +-1): the FP32
    factor of Ha, the low-rank correction for W, FP64 refinement against H.
    Returns (info_factor, info_capacitance, status, x, iters, backward_error,
    xs) with xs the solutions of extra_rhs (same factor and correction)."""
    m = H.shape[0]
    k = Wt.shape[1]
    wb = _lib().spsvm_mixed_work_bytes(m)
    work = torch.empty(max(256, wb), dtype=torch.uint8, device=H.device)
    info = torch.zeros(2, dtype=torch.int32, device=H.device)
    check(_lib().spsvm_cholesky_mixed(ptr(Ha), m, Ha.stride(0), 0.0, ptr(info), ptr(work), wb,
                                      stream_ptr()), "spsvm_cholesky_mixed")
    x = torch.zeros(m, dtype=torch.float64, device=H.device)
    if int(info[0].item()) != 0:
        return int(info[0].item()), None, None, x, 0, None, []
    lb = _lib().spsvm_lowrank_work_bytes(m, k)
    lw = torch.empty(max(256, lb), dtype=torch.uint8, device=H.device)
    check(_lib().spsvm_lowrank_factor(ptr(work), wb, m, ptr(Wt), Wt.stride(0), ptr(sign), k,
                                      ptr(lw), lb, ptr(info[1:]), stream_ptr()),
          "spsvm_lowrank_factor")
    ic = int(info[1].item())
    if ic != 0:
        return 0, ic, None, x, 0, None, []
    out = []
    for rhs in (b,) + tuple(extra_rhs):
        xx = torch.zeros(m, dtype=torch.float64, device=H.device)
        it = C.c_int32()
        be = C.c_double()
        st = _lib().spsvm_solve_lowrank(ptr(H), m, H.stride(0), ptr(rhs), ptr(xx), int(max_iter),
                                        float(tol), C.byref(it), C.byref(be), ptr(work), wb,
                                        ptr(lw), lb, k, stream_ptr())
        if st not in (L.SPSVM_OK, L.SPSVM_ERR_NO_CONVERGE):
            check(st, "spsvm_solve_lowrank")
        out.append((st, xx, it.value, be.value))
    st, x, its, be = out[0]
    return 0, 0, st, x, its, be, [o[1] for o in out[1:]]


def spsvm_active_diff(K: KMat, active, ref, kmax, rows=None):
    """(k, Wt, sign): the points whose flag differs between active and ref,
    in increasing order, their kernel rows (Wt[j, r] = K[j, D_r]) and signs
    (+1 entered, -1 left); Wt and sign are filled when k <= kmax."""
    ks = K.struct(rows)
    sb = _lib().spsvm_compact_scratch_bytes(K.n, 0)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=K.buf.device)
    ldw = max(1, kmax)
    Wt = torch.zeros((ks.rows, ldw), dtype=torch.float32, device=K.buf.device)
    sign = torch.zeros(ldw, dtype=torch.float32, device=K.buf.device)
    kd = torch.zeros(1, dtype=torch.int32, device=K.buf.device)
    check(_lib().spsvm_active_diff(C.byref(ks), ptr(active), ptr(ref), int(kmax), ptr(Wt), ldw,
                                   ptr(sign), ptr(kd), ptr(scratch), sb, stream_ptr()),
          "spsvm_active_diff")
    k = int(kd.item())
    return k, Wt[:, :min(k, kmax)], sign[:min(k, kmax)]


def spsvm_cholesky_mixed(H: torch.Tensor, shift=0.0):
    """FP32 Cholesky factor of H + shift I (H FP64, full symmetric, not
    overwritten).  Returns (info, L): L is the m x round_up(m, 4) FP32 view
    of the work buffer whose lower triangle holds the factor."""
    m = H.shape[0]
    wb = _lib().spsvm_mixed_work_bytes(m)
    work = torch.empty(max(256, wb), dtype=torch.uint8, device=H.device)
    info = torch.zeros(1, dtype=torch.int32, device=H.device)
    check(_lib().spsvm_cholesky_mixed(ptr(H), m, H.stride(0), float(shift), ptr(info), ptr(work),
                                      wb, stream_ptr()), "spsvm_cholesky_mixed")
    ldl = (m + 3) // 4 * 4
    return int(info.item()), work[:m * ldl * 4].view(torch.float32).view(m, ldl)


def spsvm_cholesky_solve(Lf: torch.Tensor, b: torch.Tensor):
    wb = _lib().spsvm_cholesky_solve_work_bytes(Lf.shape[0])
    work = torch.empty(max(16, wb), dtype=torch.uint8, device=Lf.device)
    check(_lib().spsvm_cholesky_solve(ptr(Lf), Lf.shape[0], Lf.stride(0), ptr(b), ptr(work), wb,
                                      stream_ptr()),
          "spsvm_cholesky_solve")
    return b


def spsvm_line_search(o, u, y, d, J, lam):
    n = o.numel()
    sb = _lib().spsvm_line_scratch_bytes(n)
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=o.device)
    t = C.c_double(0.0)
    check(_lib().spsvm_line_search(ptr(o), ptr(u), ptr(y), n, ptr(d), ptr(J), int(J.numel()),
                                   float(lam), C.byref(t), None, ptr(scratch), sb, stream_ptr()),
          "spsvm_line_search")
    return t.value


def spsvm_decision(B, beta, Q, gamma, precision="fp32"):
    m, d = B.shape
    nq = Q.shape[0]
    out = torch.empty(nq, dtype=torch.float32, device=Q.device)
    sb = _lib().spsvm_decision_scratch_bytes(nq, m, d, _prec(precision))
    scratch = torch.empty(max(1, sb), dtype=torch.uint8, device=Q.device)
    check(_lib().spsvm_decision(ptr(B), m, B.stride(0), ptr(beta), ptr(Q), nq, Q.stride(0), d,
                                float(gamma), _prec(precision), ptr(out), ptr(scratch), sb,
                                stream_ptr()), "spsvm_decision")
    return out


def spsvm_draw_candidates(n, J, kappa, seed, round_index):
    J = np.ascontiguousarray(np.asarray(J, dtype=np.int64))
    out = np.empty(max(1, kappa), dtype=np.int64)
    k = _lib().spsvm_draw_candidates(int(n), J.ctypes.data if len(J) else None, len(J), int(kappa),
                                     C.c_uint64(int(seed) & ((1 << 64) - 1)),
                                     C.c_uint32(int(round_index) & 0xFFFFFFFF), out.ctypes.data)
    if k < 0:
        raise ValueError("spsvm_draw_candidates: bad arguments")
    return out[:k].copy()


# ---------------------------------------------------------------- fit/predict
def make_options(candidates=256, add_per_round=64, max_newton=50, precision="fp32",
                 growth_tol=0.0, rel_tol=0.0, seed=0, initial_basis=None, fixed_basis=False,
                 refine=0, record=False, stream=None, newton_solver="mixed", score="heuristic",
                 bias=False, lowrank=False):
    o = spsvm_options()
    o.candidates = int(candidates)
    o.add_per_round = int(add_per_round)
    o.max_newton = int(max_newton)
    o.precision = _prec(precision)
    o.growth_tol = float(growth_tol)
    o.rel_tol = float(rel_tol)
    o.seed = int(seed) & ((1 << 64) - 1)
    keep = None
    if initial_basis is not None and len(initial_basis):
        keep = np.ascontiguousarray(np.asarray(initial_basis, dtype=np.int64))
        o.initial_basis = keep.ctypes.data_as(C.POINTER(C.c_int64))
        o.n_initial = len(keep)
    o.fixed_basis = int(bool(fixed_basis))
    o.refine = int(refine)
    o.record = int(bool(record))
    o.stream = stream_ptr(stream) if torch.cuda.is_available() else None
    o.newton_solver = {"mixed": L.SPSVM_SOLVE_MIXED, "fp64": L.SPSVM_SOLVE_FP64}[newton_solver]
    o.score = {"heuristic": L.SPSVM_SCORE_HEURISTIC, "exact": L.SPSVM_SCORE_EXACT}[score]
    o.bias = int(bool(bias))
    o.lowrank = int(bool(lowrank))
    return o, keep


class Model:
    """Owns an spsvm_model handle."""

    def __init__(self, handle, status):
        self.handle = C.c_void_p(handle)
        self.status = status

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                _lib().spsvm_free(self.handle)
                self.handle = C.c_void_p(None)
        except Exception:
            pass

    def info(self):
        nb = C.c_int32()
        d = C.c_int64()
        g = C.c_float()
        lam = C.c_double()
        obj = C.c_double()
        steps = C.c_int32()
        rounds = C.c_int32()
        st = C.c_int32()
        check(_lib().spsvm_model_info(self.handle, C.byref(nb), C.byref(d), C.byref(g),
                                      C.byref(lam), C.byref(obj), C.byref(steps), C.byref(rounds),
                                      C.byref(st)), "spsvm_model_info")
        return dict(n_basis=nb.value, d=d.value, gamma=g.value, lam=lam.value,
                    objective=obj.value, newton_steps=steps.value, rounds=rounds.value,
                    status=st.value)

    def bias(self):
        b = C.c_double()
        check(_lib().spsvm_model_bias(self.handle, C.byref(b)), "spsvm_model_bias")
        return b.value

    def basis_and_beta(self):
        nb = self.info()["n_basis"]
        J = np.empty(max(1, nb), dtype=np.int64)
        beta = np.empty(max(1, nb), dtype=np.float64)
        check(_lib().spsvm_model_get(self.handle, J.ctypes.data, beta.ctypes.data),
              "spsvm_model_get")
        return J[:nb], beta[:nb]

    def history(self):
        cnt = C.c_int32()
        check(_lib().spsvm_model_history(self.handle, None, 0, C.byref(cnt)), "spsvm_model_history")
        arr = (spsvm_step * max(1, cnt.value))()
        check(_lib().spsvm_model_history(self.handle, C.cast(arr, C.c_void_p), cnt.value,
                                         C.byref(cnt)), "spsvm_model_history")
        return [dict(basis=a.basis, active=a.active, gnorm=a.gnorm, t=a.t, loss=a.loss,
                     errors=a.errors, jitter=a.jitter, changed=a.changed, solve=a.solve)
                for a in arr[:cnt.value]]

    def round(self, r):
        nc = C.c_int32()
        nch = C.c_int32()
        check(_lib().spsvm_model_round(self.handle, int(r), None, C.byref(nc), None, C.byref(nch)),
              "spsvm_model_round")
        cand = np.empty(max(1, nc.value), dtype=np.int64)
        ch = np.empty(max(1, nch.value), dtype=np.int64)
        check(_lib().spsvm_model_round(self.handle, int(r), cand.ctypes.data, C.byref(nc),
                                       ch.ctypes.data, C.byref(nch)), "spsvm_model_round")
        return cand[:nc.value], ch[:nch.value]

    def device_bytes(self):
        return int(_lib().spsvm_model_device_bytes(self.handle))

    def outputs(self, n):
        o = np.empty(n, dtype=np.float32)
        check(_lib().spsvm_model_outputs(self.handle, o.ctypes.data, int(n)), "spsvm_model_outputs")
        return o

    def predict(self, Xq: torch.Tensor, stream=None):
        return spsvm_predict(self, Xq, stream)


def spsvm_fit_workspace_bytes(n, d, budget, options):
    return _lib().spsvm_fit_workspace_bytes(int(n), int(d), int(budget), C.byref(options))


def spsvm_fit(X: torch.Tensor, y: torch.Tensor, gamma, lam, budget, tol=1e-6, workspace=None,
              **opts):
    """Trains SP-SVM on device tensors X (n x d float32) and y (n float32
    in {-1,+1}); the workspace is a torch uint8 CUDA tensor (allocated here
    when not given)."""
    _require_cuda(X, y)
    assert X.dtype == torch.float32 and y.dtype == torch.float32 and X.stride(1) == 1
    n, d = X.shape
    o, keep = make_options(**opts)
    wsb = _lib().spsvm_fit_workspace_bytes(n, d, int(budget), C.byref(o))
    if workspace is None:
        workspace = torch.empty(max(1, wsb), dtype=torch.uint8, device=X.device)
    handle = C.c_void_p()
    rc = _lib().spsvm_fit(ptr(X), n, d, X.stride(0), ptr(y), float(gamma), float(lam), int(budget),
                          float(tol), C.byref(o), ptr(workspace), workspace.numel(),
                          C.byref(handle))
    del keep
    if rc not in (L.SPSVM_OK, L.SPSVM_ERR_NO_CONVERGE):
        check(rc, "spsvm_fit")
    return Model(handle.value, rc)


def spsvm_predict_work_bytes(model: Model, nq: int) -> int:
    """Device work bytes one spsvm_predict_ws call on nq queries needs."""
    return int(_lib().spsvm_predict_work_bytes(model.handle, int(nq)))


def spsvm_predict(model: Model, Xq: torch.Tensor, stream=None, work=None):
    """Decision values of the model on the query rows Xq.  work: optional
    device uint8 tensor of at least spsvm_predict_work_bytes(model, nq)
    bytes (the library otherwise takes its work memory stream-ordered)."""
    _require_cuda(Xq)
    assert Xq.dtype == torch.float32 and Xq.stride(1) == 1
    out = torch.empty(Xq.shape[0], dtype=torch.float32, device=Xq.device)
    if work is None:
        check(_lib().spsvm_predict(model.handle, ptr(Xq), Xq.shape[0], Xq.stride(0), ptr(out),
                                   stream_ptr(stream)), "spsvm_predict")
    else:
        assert work.dtype == torch.uint8 and work.is_cuda
        check(_lib().spsvm_predict_ws(model.handle, ptr(Xq), Xq.shape[0], Xq.stride(0), ptr(out),
                                      ptr(work), work.numel(), stream_ptr(stream)),
              "spsvm_predict_ws")
    return out


# ---------------------------------------------------------------- batched / serving
def spsvm_fit_batched(X: torch.Tensor, problems, workers=4, **opts):
    """problems: list of dicts with rows (int64 array or None), y (float32
    array), gamma, lam, budget, tol, seed.  Returns (models, statuses)."""
    _require_cuda(X)
    n, d = X.shape
    keep = []
    arr = (spsvm_problem * max(1, len(problems)))()
    for k, p in enumerate(problems):
        rows = p.get("rows")
        y = np.ascontiguousarray(np.asarray(p["y"], dtype=np.float32))
        keep.append(y)
        q = arr[k]
        if rows is not None:
            rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
            keep.append(rows)
            q.rows = rows.ctypes.data
            q.n_rows = len(rows)
        else:
            q.rows = None
            q.n_rows = n
        q.y = y.ctypes.data
        q.gamma = float(p["gamma"])
        q.lambda_ = float(p["lam"])
        q.basis_budget = int(p["budget"])
        q.tol = float(p.get("tol", 1e-6))
        q.seed = int(p.get("seed", 0))
    o, k0 = make_options(**opts)
    outs = (C.c_void_p * max(1, len(problems)))()
    st = (C.c_int32 * max(1, len(problems)))()
    rc = _lib().spsvm_fit_batched(ptr(X), n, d, X.stride(0), arr, len(problems), C.byref(o),
                                  int(workers), C.cast(outs, C.c_void_p), C.cast(st, C.c_void_p))
    del keep, k0
    models = [Model(outs[k], st[k]) if outs[k] else None for k in range(len(problems))]
    if rc != L.SPSVM_OK and all(m is None for m in models):
        check(rc, "spsvm_fit_batched")
    return models, [st[k] for k in range(len(problems))]


def spsvm_fit_ovo(X: torch.Tensor, labels, classes, gamma, lam, budget, tol=1e-6, workers=4,
                  **opts):
    """One-vs-one: one binary model per class pair (a, b), a < b, in the order
    (0,1), (0,2), ..., fitted as one batch on the device X (n x d float32);
    labels: host ints in [0, classes).  Returns (models, statuses)."""
    _require_cuda(X)
    assert X.dtype == torch.float32 and X.stride(1) == 1
    n, d = X.shape
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    assert lab.shape == (n,)
    P = classes * (classes - 1) // 2
    o, keep = make_options(**opts)
    outs = (C.c_void_p * max(1, P))()
    st = (C.c_int32 * max(1, P))()
    rc = _lib().spsvm_fit_ovo(ptr(X), n, d, X.stride(0), lab.ctypes.data, int(classes),
                              float(gamma), float(lam), int(budget), float(tol), C.byref(o),
                              int(workers), C.cast(outs, C.c_void_p), C.cast(st, C.c_void_p))
    del keep
    models = [Model(outs[k], st[k]) if outs[k] else None for k in range(P)]
    if rc != L.SPSVM_OK and all(m is None for m in models):
        check(rc, "spsvm_fit_ovo")
    return models, [st[k] for k in range(P)]


def spsvm_predict_ovo(models, classes, Xq: torch.Tensor, votes=False, stream=None):
    """Labels (device int32) of the queries by one-vs-one voting over the pair
    models of spsvm_fit_ovo; with votes=True also the nq x classes vote
    counts."""
    _require_cuda(Xq)
    assert Xq.dtype == torch.float32 and Xq.stride(1) == 1
    nq = Xq.shape[0]
    P = classes * (classes - 1) // 2
    arr = (C.c_void_p * max(1, P))(*[m.handle.value for m in models])
    wb = _lib().spsvm_predict_ovo_work_bytes(int(classes), nq)
    work = torch.empty(max(256, wb), dtype=torch.uint8, device=Xq.device)
    lab = torch.empty(max(1, nq), dtype=torch.int32, device=Xq.device)
    vt = torch.empty((max(1, nq), classes), dtype=torch.int32, device=Xq.device) if votes else None
    check(_lib().spsvm_predict_ovo(C.cast(arr, C.c_void_p), int(classes), ptr(Xq), nq, Xq.stride(0),
                                   ptr(lab), ptr(vt), ptr(work), wb, stream_ptr(stream)),
          "spsvm_predict_ovo")
    return (lab[:nq], vt[:nq] if vt is not None else None)


class _Borrowed(Model):
    """A model owned by the server (not freed here)."""

    def __del__(self):
        pass


class Server:
    """spsvm_server: continuous-batching request loop with HBM admission."""

    def __init__(self, hbm_budget_bytes, workers=4):
        h = C.c_void_p()
        check(_lib().spsvm_server_create(int(hbm_budget_bytes), int(workers), C.byref(h)),
              "spsvm_server_create")
        self.h = h

    def submit_fit(self, X, y, gamma, lam, budget, tol=1e-6, **opts):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
        o, keep = make_options(**opts)
        rid = C.c_int64()
        check(_lib().spsvm_server_submit_fit(self.h, X.ctypes.data, X.shape[0], X.shape[1],
                                             y.ctypes.data, float(gamma), float(lam), int(budget),
                                             float(tol), C.byref(o), C.byref(rid)),
              "spsvm_server_submit_fit")
        del keep
        return rid.value

    def submit_predict(self, fit_id, Xq):
        Xq = np.ascontiguousarray(np.asarray(Xq, dtype=np.float32))
        rid = C.c_int64()
        check(_lib().spsvm_server_submit_predict(self.h, int(fit_id), Xq.ctypes.data, Xq.shape[0],
                                                 C.byref(rid)), "spsvm_server_submit_predict")
        self._nq = getattr(self, "_nq", {})
        self._nq[rid.value] = Xq.shape[0]
        return rid.value

    def wait(self, rid, timeout_s=-1.0):
        st = C.c_int32()
        lat = C.c_double()
        check(_lib().spsvm_server_wait(self.h, int(rid), float(timeout_s), C.byref(st),
                                       C.byref(lat)), "spsvm_server_wait")
        return st.value, lat.value

    def decision(self, rid):
        nq = self._nq[rid]
        out = np.empty(nq, dtype=np.float32)
        check(_lib().spsvm_server_result(self.h, int(rid), out.ctypes.data, nq, None),
              "spsvm_server_result")
        return out

    def model(self, rid):
        m = C.c_void_p()
        check(_lib().spsvm_server_result(self.h, int(rid), None, 0, C.byref(m)),
              "spsvm_server_result")
        return _Borrowed(m.value, 0) if m.value else None

    def release(self, fit_id):
        check(_lib().spsvm_server_release(self.h, int(fit_id)), "spsvm_server_release")

    def stats(self):
        a, b = C.c_int64(), C.c_int64()
        c, d = C.c_size_t(), C.c_size_t()
        check(_lib().spsvm_server_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
              "spsvm_server_stats")
        return dict(done=a.value, queued=b.value, hbm_in_use=c.value, hbm_peak=d.value)

    def close(self):
        if self.h and self.h.value:
            _lib().spsvm_server_destroy(self.h)
            self.h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
