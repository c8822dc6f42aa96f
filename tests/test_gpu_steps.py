"""Step-by-step parity of the CUDA path against the float64 oracle, element
by element, on seeded inputs that span several tiles with ragged tails.
Each step is fed the same inputs on both sides (for the HBM passes the
oracle's own kernel matrix, rounded to the stored format), so that only the
step under test differs.

Tolerances (derived from the arithmetic, stated per test):
  * kernel values: FP32 form, |dK| <= 2e-6 + 4 eps32 gamma (|x|^2+|z|^2);
    BF16SPLIT form, the three-term split is exact for FP32 operands and the
    three dropped products are below 2^-24 |x z| each, so the dot product
    carries FP32 rounding of its 6 d products accumulated in FP32:
    |dK| <= 2e-6 + 8 eps32 gamma (|x|^2 + |z|^2).
  * sums of n products in FP32 with FP64 promotion every 32 terms:
    |err| <= 1e-5 * sum |terms|.
  * FP64 Cholesky / solves: backward-stable, 1e-10 relative.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import spsvm as O

pytestmark = pytest.mark.gpu

# kernel-value bound of the split form, relative to gamma (|x|^2 + |z|^2)
KTOL_SPLIT = 8 * 2 ** -24

DEV = "cuda"


def _data(n, d, seed, scale=1.0):
    g = np.random.default_rng(seed)
    X = (g.standard_normal((n, d)) * scale + 0.3).astype(np.float32)
    y = np.where(g.random(n) < 0.5, 1.0, -1.0).astype(np.float32)
    return X, y


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t if dtype is None else t.to(dtype)


def _store(K_rows, fmt, sp):
    """Loads a (rows x n) float64 matrix into a KMat of the given format."""
    rows, n = K_rows.shape
    km = sp.kmat_empty(n, rows, fmt)
    ld = km.ld
    K32 = torch.from_numpy(K_rows.astype(np.float32)).to(DEV)
    if fmt == "fp32":
        km.buf.view(-1)[: rows * ld].view(rows, ld)[:, :n] = K32
        ref = K32.double()
    else:
        hi = K32.to(torch.bfloat16)
        lo = (K32 - hi.float()).to(torch.bfloat16)
        km.buf.view(-1)[: rows * ld].view(rows, ld)[:, :n] = hi
        km.buf.view(-1)[km.plane: km.plane + rows * ld].view(rows, ld)[:, :n] = lo
        ref = hi.double() + lo.double()
    return km, ref.cpu().numpy()


@pytest.fixture(scope="module")
def sp():
    import paper_1404_1066_gb300 as sp
    sp.load()
    return sp


@pytest.mark.parametrize("n,d,m", [(1000, 20, 70), (257, 37, 64), (130, 5, 1), (3000, 130, 129),
                                   (290, 64, 200)])
@pytest.mark.parametrize("prec,store", [("fp32", "fp32"), ("fp32", "bf16split"), ("bf16split", "fp32")])
def test_kernel_block(sp, n, d, m, prec, store):
    """Arithmetic form x storage format (the tensor-core form stores FP32);
    the stored hi + lo planes add 2^-17 relative rounding of each value."""
    X, _ = _data(n, d, 1)
    gamma = 1.0 / d
    g = np.random.default_rng(2)
    idx = g.choice(n, size=m, replace=False).astype(np.int64)
    P = sp.spsvm_prepare_points(_t(X), prec)
    nrm = P.norms.cpu().numpy()
    np.testing.assert_allclose(nrm, (X.astype(np.float64) ** 2).sum(1), rtol=1e-6)
    km = sp.kmat_empty(n, m + 3, store)
    sp.spsvm_kernel_block(P, _t(idx), gamma, prec, km, row0=3)
    torch.cuda.synchronize()
    got = km.to_float().cpu().numpy().astype(np.float64)[3:]
    ref = O.rbf_kernel(X, X[idx], gamma).T
    sq = (X.astype(np.float64) ** 2).sum(1)
    scale = gamma * (sq[None, :] + sq[idx][:, None])
    tol = (4 * 2 ** -24 if prec == "fp32" else KTOL_SPLIT) * scale + 2e-6
    if store == "bf16split":
        tol = tol + 2.0 ** -17 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)
    # rows before row0 untouched
    assert float(km.to_float()[:3].abs().max()) == 0.0


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
def test_score_candidates(sp, prec):
    n, d = 2100, 24
    X, y = _data(n, d, 3)
    gamma, lam = 1.0 / d, 1e-3
    g = np.random.default_rng(4)
    J = g.choice(n, size=40, replace=False)
    beta = g.standard_normal(40) * 0.3
    o = (O.rbf_kernel(X, X[J], gamma) @ beta).astype(np.float32).astype(np.float64)
    pool = np.setdiff1d(np.arange(n), J)
    cand = g.choice(pool, size=100, replace=False).astype(np.int64)
    P = sp.spsvm_prepare_points(_t(X), prec)
    gg, hh, dd = sp.spsvm_score_candidates(P, _t(y), _t(o.astype(np.float32)), _t(cand), gamma,
                                           lam, prec)
    # oracle with o as given (the reg term lambda k_cJ beta is o_c)
    delta, gr, hr = O.score_candidates(X, y.astype(np.float64), list(J), beta, o, cand, gamma, lam)
    gr = lam * o[cand] + (gr - lam * (O.rbf_kernel(X[cand], X[J], gamma) @ beta))
    delta = gr * gr / (2 * hr)
    S = y * o < 1
    res = np.where(S, o - y, 0)
    Kc = O.rbf_kernel(X, X[cand], gamma)
    gabs = np.abs(res) @ Kc + lam * np.abs(o[cand])
    ktol = 4 * 2 ** -24 if prec == "fp32" else KTOL_SPLIT
    sq = (X.astype(np.float64) ** 2).sum(1)
    kerr = ktol * gamma * (sq.max() + sq.max()) + 2e-6
    gtol = 1e-5 * gabs + kerr * np.abs(res).sum()
    htol = 1e-5 * hr + 2 * kerr * S.sum()
    assert np.all(np.abs(gg.cpu().numpy() - gr) <= gtol)
    assert np.all(np.abs(hh.cpu().numpy() - hr) <= htol)
    # ranking agrees wherever the scores are separated by more than the error
    dg = dd.cpu().numpy()
    rel = np.abs(dg - delta) / delta
    assert np.all(rel <= 2 * (gtol / np.abs(gr) + htol / hr) + 1e-12)


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
def test_score_candidates_exact(sp, prec):
    """Exact one-dimensional scores against the oracle's (exact line search
    along each new coefficient, float64, direct differences) on the same o.
    The kernel-value errors bound the errors of g and h as for the heuristic
    score; delta moves by at most |t| dg + t^2 dh / 2 (plus FP32 summation),
    and t by (dg + |t| dh) / h."""
    n, d = 2100, 24
    X, y = _data(n, d, 3)
    gamma, lam = 1.0 / d, 1e-3
    g = np.random.default_rng(4)
    J = g.choice(n, size=40, replace=False)
    beta = g.standard_normal(40) * 0.3
    o = (O.rbf_kernel(X, X[J], gamma) @ beta).astype(np.float32).astype(np.float64)
    pool = np.setdiff1d(np.arange(n), J)
    cand = g.choice(pool, size=100, replace=False).astype(np.int64)
    P = sp.spsvm_prepare_points(_t(X), prec)
    dd, tt = sp.spsvm_score_candidates_exact(P, _t(y), _t(o.astype(np.float32)), _t(cand), gamma,
                                             lam, prec)
    dg, tg = dd.cpu().numpy(), tt.cpu().numpy()
    dref, tref = O.score_candidates_exact(X, y.astype(np.float64), list(J), beta, o, cand, gamma, lam)
    _, gr, hr = O.score_candidates(X, y.astype(np.float64), list(J), beta, o, cand, gamma, lam)
    S = y * o < 1
    res = np.where(S, o - y, 0)
    Kc = O.rbf_kernel(X, X[cand], gamma)
    ktol = 4 * 2 ** -24 if prec == "fp32" else KTOL_SPLIT
    sq = (X.astype(np.float64) ** 2).sum(1)
    kerr = ktol * gamma * 2 * sq.max() + 2e-6
    gtol = 1e-5 * (np.abs(res) @ Kc + lam * np.abs(o[cand])) + kerr * (np.abs(res).sum() + n)
    htol = 1e-5 * hr + 2 * kerr * n
    loss0 = 0.5 * np.sum(np.where(S, 1 - y * o, 0) ** 2)
    dtol = np.abs(tref) * gtol + 0.5 * tref ** 2 * htol + 1e-5 * np.abs(dref) + 1e-6 * loss0 / n
    assert np.all(dg >= 0)
    assert np.all(np.abs(dg - dref) <= dtol), float(np.max(np.abs(dg - dref) / dtol))
    ttol = 2 * (gtol + np.abs(tref) * htol) / hr + 1e-6 * np.abs(tref)
    assert np.all(np.abs(tg - tref) <= ttol), float(np.max(np.abs(tg - tref) / ttol))


@pytest.mark.parametrize("fmt", ["fp32", "bf16split"])
@pytest.mark.parametrize("n,m", [(1000, 70), (4099, 129), (33, 1)])
def test_outputs_gemv(sp, fmt, n, m):
    g = np.random.default_rng(5)
    K = np.exp(-g.random((m, n)) * 3)
    km, Kref = _store(K, fmt, sp)
    beta = g.standard_normal(m)
    y = np.where(g.random(n) < 0.5, 1.0, -1.0).astype(np.float32)
    o = torch.zeros(n, dtype=torch.float32, device=DEV)
    active, stats = sp.spsvm_outputs(km, _t(beta), _t(y), o)
    torch.cuda.synchronize()
    o_ref = Kref.T @ beta
    og = o.cpu().numpy().astype(np.float64)
    tol = 1e-6 * (np.abs(Kref.T) @ np.abs(beta)) + 1e-7 * np.abs(o_ref)
    assert np.all(np.abs(og - o_ref) <= tol)
    # flags, loss and errors from the GPU's own o (same precision decides)
    margin = y.astype(np.float32) * o.cpu().numpy()
    np.testing.assert_array_equal(active.cpu().numpy(), (margin < 1).astype(np.uint8))
    st = stats.cpu().numpy()
    xi = np.maximum(0, 1 - margin.astype(np.float64))
    assert st[0] == pytest.approx(0.5 * np.sum(xi ** 2), rel=1e-12)
    assert st[1] == np.sum(margin <= 0)
    assert st[2] == np.sum(margin < 1)
    u = torch.empty(n, dtype=torch.float32, device=DEV)
    v = g.standard_normal(m)
    sp.spsvm_gemv(km, _t(v), u)
    torch.cuda.synchronize()
    u_ref = Kref.T @ v
    assert np.all(np.abs(u.cpu().numpy() - u_ref) <= 1e-6 * (np.abs(Kref.T) @ np.abs(v)) + 1e-7 * np.abs(u_ref))
    sp.spsvm_gemv(km, _t(v), u, accumulate=True)
    torch.cuda.synchronize()
    assert np.all(np.abs(u.cpu().numpy() - 2 * u_ref) <= 4e-6 * (np.abs(Kref.T) @ np.abs(v)) + 2e-7 * np.abs(u_ref))


def _split_ref(K):
    """hi + lo of FP32 values, as the compaction splits them (float64)."""
    K32 = torch.from_numpy(np.asarray(K, dtype=np.float32))
    hi = K32.to(torch.bfloat16)
    lo = (K32 - hi.float()).to(torch.bfloat16)
    return (hi.double() + lo.double()).numpy()


@pytest.mark.parametrize("fmt,kc_fmt", [("fp32", "fp32"), ("bf16split", "bf16split"), ("fp32", "bf16split")])
# few active points (at most n / 64) take the gather path, more the scan
@pytest.mark.parametrize("n,m,p", [(5000, 70, 0.5), (1000, 8, 0.0), (1000, 9, 1.0), (777, 64, 0.03),
                                   (20000, 70, 0.01), (50000, 130, 0.005), (6400, 20, 0.018)])
def test_compact_and_masked_products(sp, fmt, kc_fmt, n, m, p):
    g = np.random.default_rng(6)
    K = np.exp(-g.random((m, n)) * 3)
    km, Kref = _store(K, fmt, sp)
    act = (g.random(n) < p).astype(np.uint8)
    w1 = g.standard_normal(n).astype(np.float32)
    w2 = g.standard_normal(n).astype(np.float32)
    kc = sp.kmat_empty(km.ld, m, kc_fmt, ld=km.ld)
    a, b, nact, pos = sp.spsvm_compact_active(km, _t(act), _t(w1), _t(w2), kc)
    torch.cuda.synchronize()
    S = act.astype(bool)
    ns = int(S.sum())
    assert int(nact.item()) == ns
    np.testing.assert_array_equal(pos.cpu().numpy()[S], np.arange(ns))
    # the compacted rows are exact copies (or the exact hi / lo split of the
    # FP32 values); the tail to a multiple of 128 is zero
    kcf = kc.to_float().cpu().numpy().astype(np.float64)
    want = Kref[:, S] if fmt == kc_fmt else _split_ref(Kref[:, S])
    np.testing.assert_array_equal(kcf[:, :ns], want)
    tail = ((ns + 127) // 128) * 128
    assert np.all(kcf[:, ns:tail] == 0)
    ra = Kref[:, S] @ w1[S].astype(np.float64)
    rb = Kref[:, S] @ w2[S].astype(np.float64)
    tola = 1e-6 * (np.abs(Kref[:, S]) @ np.abs(w1[S])) + 1e-12
    tolb = 1e-6 * (np.abs(Kref[:, S]) @ np.abs(w2[S])) + 1e-12
    assert np.all(np.abs(a.cpu().numpy() - ra) <= tola)
    assert np.all(np.abs(b.cpu().numpy() - rb) <= tolb)


@pytest.mark.parametrize("prec,kfmt", [("fp32", "fp32"), ("bf16split", "bf16split"), ("bf16split", "fp32")])
@pytest.mark.parametrize("n,m,p", [(9000, 70, 0.6), (20000, 130, 0.5), (300, 64, 1.0), (2000, 1, 0.7)])
def test_gram(sp, prec, kfmt, n, m, p):
    """The BF16SPLIT Gram matrix reads the compact copy as hi / lo planes, from
    K stored as planes or (the fit's layout) in FP32 and split on the way."""
    g = np.random.default_rng(7)
    n_all = n
    X, _ = _data(n_all, 12, 8)
    J = g.choice(n_all, size=m, replace=False)
    K = O.rbf_kernel(X, X[J], 1.0 / 12).T          # rows = basis
    km, Kref = _store(K, kfmt, sp)
    act = (g.random(n) < p).astype(np.uint8)
    kc = sp.kmat_empty(km.ld, m, prec, ld=km.ld)
    _, _, nact, _ = sp.spsvm_compact_active(km, _t(act), None, None, kc)
    lam = 1e-3
    H = sp.spsvm_gram(kc, nact, n, km, _t(J.astype(np.int64)), lam, prec)
    torch.cuda.synchronize()
    S = act.astype(bool)
    KS = Kref[:, S]
    KJJ = Kref[:, J].T
    Href = lam * 0.5 * (KJJ + KJJ.T) + KS @ KS.T
    Hg = H.cpu().numpy()
    np.testing.assert_array_equal(Hg, Hg.T)
    bound = np.abs(KS) @ np.abs(KS).T
    # BF16SPLIT: the hi+lo kernel values carry ~2^-17 relative error, plus
    # tensor-core FP32 accumulation
    rel = 1e-5 if prec == "fp32" else 1e-4
    assert np.all(np.abs(Hg - Href) <= rel * bound + 1e-12), np.max(np.abs(Hg - Href) / (bound + 1e-30))


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("m", [1, 5, 63, 64, 65, 200, 513, 1500])
def test_cholesky_and_solve(sp, m, tc):
    g = np.random.default_rng(m)
    A = g.standard_normal((m, m + 3))
    H = A @ A.T + 1e-2 * np.eye(m)
    Ht = _t(H.copy())
    info = sp.spsvm_cholesky(Ht, tensor_cores=tc)
    assert info == 0
    Lg = np.tril(Ht.cpu().numpy())
    Lr = np.linalg.cholesky(H)
    np.testing.assert_allclose(Lg, Lr, rtol=1e-9, atol=1e-12 * np.abs(Lr).max())
    b = g.standard_normal(m)
    bt = _t(b.copy())
    sp.spsvm_cholesky_solve(Ht, bt)
    x = bt.cpu().numpy()
    xr = np.linalg.solve(H, b)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr) * max(1, np.linalg.cond(H) * 1e-6)


@pytest.mark.parametrize("m", [2, 64, 127, 4100])
def test_solve_padded_rows_and_reused_work(sp, m):
    """Row pitch larger than m, a ragged last block, and several solves with
    the same factor and the same work buffer (the flags are reset per call)."""
    g = np.random.default_rng(m + 1)
    A = g.standard_normal((m, m + 5)) / np.sqrt(m)
    H = A @ A.T + 0.5 * np.eye(m)
    big = np.zeros((m, m + 37))
    big[:, :m] = H
    Hb = _t(big)
    Hv = Hb[:, :m]
    assert Hv.stride(0) == m + 37
    assert sp.spsvm_cholesky(Hv) == 0
    lib = sp.load()
    wb = lib.spsvm_cholesky_solve_work_bytes(m)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    for k in range(3):
        b = g.standard_normal(m)
        bt = _t(b.copy())
        rc = lib.spsvm_cholesky_solve(Hv.data_ptr(), m, m + 37, bt.data_ptr(), work.data_ptr(),
                                      wb, None)
        assert rc == 0
        torch.cuda.synchronize()
        code = ctypes.c_int32(-9)
        assert lib.spsvm_device_status(ctypes.byref(code)) == 0 and code.value == 0
        xr = np.linalg.solve(H, b)
        np.testing.assert_allclose(bt.cpu().numpy(), xr, rtol=1e-10, atol=1e-12 * np.abs(xr).max())
    # too small a work buffer is refused before any launch
    rc = lib.spsvm_cholesky_solve(Hv.data_ptr(), m, m + 37, bt.data_ptr(), work.data_ptr(),
                                  wb - 1, None)
    assert rc == -2


@pytest.mark.parametrize("shift", [0.0, 0.3])
@pytest.mark.parametrize("m", [1, 63, 64, 65, 300, 1500])
def test_mixed_solve_reaches_fp64_backward_error(sp, m, shift):
    """FP32 factor + FP64 refinement: (H + shift I) x = b to a normwise
    backward error <= 1e-13 (an FP64 Cholesky solve reaches ~1e-16..1e-14),
    with H left bit-unchanged."""
    g = np.random.default_rng(m + 7)
    A = g.standard_normal((m, m + 3)) / np.sqrt(m)
    H = A @ A.T + 1e-2 * np.eye(m)
    b = g.standard_normal(m)
    Ht = _t(H.copy())
    info, st, x, iters, be = sp.spsvm_solve_mixed(Ht, _t(b.copy()), shift=shift)
    assert info == 0 and st == 0, (info, st, iters, be)
    np.testing.assert_array_equal(Ht.cpu().numpy(), H)
    xs = x.cpu().numpy()
    Hs = H + shift * np.eye(m)
    r = b - Hs @ xs
    ref_be = np.max(np.abs(r)) / (np.max(np.abs(Hs).sum(1)) * np.max(np.abs(xs)) + np.max(np.abs(b)))
    assert ref_be <= 1e-13 and be <= 1e-13, (ref_be, be, iters)
    xr = np.linalg.solve(Hs, b)
    assert np.linalg.norm(xs - xr) <= 1e-10 * np.linalg.norm(xr) * max(1.0, np.linalg.cond(Hs) * 1e-4)


@pytest.mark.parametrize("m", [1, 63, 64, 65, 200, 1000, 4100])
def test_mixed_factor_meets_fp32_cholesky_backward_error(sp, m):
    """The FP32 factor of H + shift I from the tiled factorisation obeys the
    componentwise backward-error bound of Cholesky in precision u = 2^-24
    (Higham, Accuracy and Stability, Thm 10.3): |L L^T - A| <= g |L| |L|^T
    with g = (m + 1) u / (1 - (m + 1) u), plus u |A| for rounding A to FP32.
    A wrong tile (a transposed operand, a missed update) breaks it by orders
    of magnitude; ragged sizes cover the identity-padded last tile."""
    g = np.random.default_rng(m)
    A = g.standard_normal((m, m + 4)) / np.sqrt(m + 4)
    H = A @ A.T + 0.05 * np.eye(m)
    shift = 0.01
    info, Lw = sp.spsvm_cholesky_mixed(_t(H), shift)
    assert info == 0
    Lf = np.tril(Lw[:, :m].cpu().numpy().astype(np.float64))
    Ash = H + shift * np.eye(m)
    u = 2.0 ** -24
    gam = (m + 1) * u / (1 - (m + 1) * u)
    bound = gam * (np.abs(Lf) @ np.abs(Lf).T) + u * np.abs(Ash)
    err = np.abs(Lf @ Lf.T - Ash)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and it is the factor: compare with the FP64 factor (condition ~ 1e2)
    R = np.linalg.cholesky(Ash)
    assert np.max(np.abs(Lf - R)) <= 1e-4 * np.max(np.abs(R))


@pytest.mark.parametrize("m", [16384, 16400])
def test_mixed_solve_large(sp, m):
    """Past 256 tile rows (more solve blocks than SMs; the last block ragged at
    16,400) the mixed solve still reaches FP64 backward error.
    H = c I + U U^T (U 64 wide) is built and checked on the device."""
    g = torch.Generator(device="cuda").manual_seed(m)
    U = torch.randn((m, 64), generator=g, dtype=torch.float64, device="cuda")
    H = U @ U.T
    H.diagonal().add_(8.0)
    b = torch.randn(m, generator=g, dtype=torch.float64, device="cuda")
    info, st, x, iters, be = sp.spsvm_solve_mixed(H, b)
    assert info == 0 and st == 0, (info, st, iters, be)
    r = b - H @ x
    bound = 1e-13 * (H.abs().sum(1).max() * x.abs().max() + b.abs().max())
    assert float(r.abs().max()) <= float(bound)
    del U, H


def test_mixed_solve_reports_fp32_breakdown_and_stagnation(sp):
    H = np.eye(100)
    H[70, 70] = -1.0
    info, st, _, _, _ = sp.spsvm_solve_mixed(_t(H), _t(np.ones(100)))
    assert info == 71 and st is None
    # condition number ~1e12: the FP32 factor either breaks down or cannot
    # refine to FP64 backward error; never a wrong "converged" answer
    g = np.random.default_rng(9)
    Q, _ = np.linalg.qr(g.standard_normal((200, 200)))
    H = (Q * np.logspace(0, -12, 200)) @ Q.T
    H = 0.5 * (H + H.T)
    b = g.standard_normal(200)
    info, st, x, iters, be = sp.spsvm_solve_mixed(_t(H), _t(b))
    if info == 0 and st == 0:
        xs = x.cpu().numpy()
        r = b - H @ xs
        assert np.max(np.abs(r)) <= 1e-13 * (np.max(np.abs(H).sum(1)) * np.max(np.abs(xs)) + np.max(np.abs(b)))
    else:
        assert info != 0 or st == -4


@pytest.mark.parametrize("tc", [False, True])
def test_cholesky_ill_conditioned_newton_matrix(sp, tc):
    # the Newton matrix of Eq. 4 on RBF data: lambda K_JJ + K_SJ^T K_SJ,
    # lambda = 1e-4, kernel rows of nearby points (condition number ~1e9)
    g = np.random.default_rng(3)
    X = g.standard_normal((3000, 8)) * 0.7
    J = np.arange(0, 3000, 3)[:900]
    K = O.rbf_kernel(X, X[J], 0.125)
    S = g.random(3000) < 0.3
    H = 1e-4 * K[J] + K[S].T @ K[S]
    H = 0.5 * (H + H.T)
    Ht = _t(H.copy())
    assert sp.spsvm_cholesky(Ht, tensor_cores=tc) == 0
    Lg = np.tril(Ht.cpu().numpy())
    # backward error of the factorisation, as FP64 Cholesky guarantees
    assert np.linalg.norm(Lg @ Lg.T - H) <= 1e-13 * np.linalg.norm(H)


def test_cholesky_reports_indefinite(sp):
    H = np.eye(100)
    H[70, 70] = -1.0
    info = sp.spsvm_cholesky(_t(H))
    assert info == 71
    assert sp.spsvm_cholesky(_t(np.zeros((3, 3)))) == 1


@pytest.mark.parametrize("seed", range(6))
def test_line_search(sp, seed):
    g = np.random.default_rng(100 + seed)
    n, m = 4000 + seed * 37, 30
    X, y = _data(n, 6, seed)
    y = y.astype(np.float64)
    J = g.choice(n, size=m, replace=False)
    KnJ = O.rbf_kernel(X, X[J], 0.2)
    KJJ = KnJ[J]
    lam = 1e-3
    beta = g.standard_normal(m) * 0.5
    o = KnJ @ beta
    S = y * o < 1
    H = lam * KJJ + KnJ[S].T @ KnJ[S]
    bb = np.linalg.solve(H, KnJ[S].T @ y[S])
    d = (bb - beta) * (1.0 if seed % 3 else 0.3)
    u = KnJ @ d
    o32 = o.astype(np.float32)
    u32 = u.astype(np.float32)
    # both sides see the FP32-rounded o and u
    t_ref = O.line_search(beta, d, o32.astype(np.float64), u32.astype(np.float64), y, KJJ, lam)
    # a0, a1 computed on the GPU from o_J, u_J: feed consistent values
    t = sp.spsvm_line_search(_t(o32), _t(u32), _t(y.astype(np.float32)), _t(d), _t(J.astype(np.int64)), lam)
    # compare through phi: the GPU step is as good as the exact minimiser
    phi = lambda s: O.objective(beta + s * d, KnJ, KJJ, y, lam)
    assert phi(t) <= phi(t_ref) + 1e-7 * abs(phi(t_ref))
    assert t == pytest.approx(t_ref, rel=2e-4, abs=1e-6)


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
@pytest.mark.parametrize("nq,m,d", [(1000, 70, 20), (129, 1, 3), (5000, 257, 64),
                                    (70001, 300, 40), (3000, 1031, 128)])
def test_decision(sp, prec, nq, m, d):
    """Decision values against the oracle's FP64 kernel: the split form on
    the tensor cores (several basis blocks, a ragged query tail, three query
    passes at nq = 70,001) within the kernel-value bound of its dot
    products plus the ex2 approximation."""
    g = np.random.default_rng(9 + m)
    B = g.standard_normal((m, d)).astype(np.float32)
    Q = g.standard_normal((nq, d)).astype(np.float32)
    beta = g.standard_normal(m)
    gamma = 0.5 / d
    out = sp.spsvm_decision(_t(B), _t(beta), _t(Q), gamma, prec)
    torch.cuda.synchronize()
    Kq = O.rbf_kernel(Q, B, gamma)
    ref = Kq @ beta
    sq = (Q.astype(np.float64) ** 2).sum(1)
    sb = (B.astype(np.float64) ** 2).sum(1)
    if prec == "fp32":
        krel = 4 * 2 ** -24 * gamma * (sq[:, None] + sb[None, :])
    else:
        krel = KTOL_SPLIT * gamma * (sq[:, None] + sb[None, :]) + 2.0 ** -21
    tol = (Kq * krel) @ np.abs(beta) + 1e-6 * (Kq @ np.abs(beta)) + 1e-7
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= tol), float(np.max(err - tol))


def test_decision_split_is_deterministic_and_work_is_private(sp):
    """The split form's predict: the caller-owned work path equals the
    stream-ordered one bit for bit, and two calls on one model from two
    streams, each with its own work, give the same values as alone."""
    g = np.random.default_rng(5)
    n, d = 6000, 32
    X = g.standard_normal((n, d)).astype(np.float32)
    y = np.where(X[:, 0] + 0.3 * X[:, 1] > 0, 1.0, -1.0).astype(np.float32)
    m = sp.spsvm_fit(_t(X), _t(y), 1.0 / d, 1e-3, 256, 1e-6, precision="bf16split",
                     candidates=128, add_per_round=64, seed=3)
    Qa = _t(g.standard_normal((40000, d)).astype(np.float32))
    Qb = _t(g.standard_normal((1234, d)).astype(np.float32))
    ra = sp.spsvm_predict(m, Qa)
    rb = sp.spsvm_predict(m, Qb)
    wa = torch.empty(sp.spsvm_predict_work_bytes(m, Qa.shape[0]), dtype=torch.uint8, device="cuda")
    wb = torch.empty(sp.spsvm_predict_work_bytes(m, Qb.shape[0]), dtype=torch.uint8, device="cuda")
    assert wa.numel() > 0 and wb.numel() > 0
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        fa = sp.spsvm_predict(m, Qa, stream=s1, work=wa)
    with torch.cuda.stream(s2):
        fb = sp.spsvm_predict(m, Qb, stream=s2, work=wb)
    torch.cuda.synchronize()
    assert torch.equal(fa, ra) and torch.equal(fb, rb)
    with pytest.raises(sp.SpsvmError):
        sp.spsvm_predict(m, Qa, work=wb[:16])


@pytest.mark.parametrize("ctas", [1, 2, 3])
def test_mixed_factor_completes_on_a_small_grid(sp, ctas):
    """The tile factorisation completes with any number of resident CTAs,
    down to one (launches on other streams may hold the rest of the GPU):
    the CTA that runs the chain of diagonal tiles takes the other tiles'
    work while it waits.  Grids of 1-3 CTAs against the full grid, on 17 and
    5 tile rows (the last one ragged), with a breakdown at a late pivot."""
    from paper_1404_1066_gb300 import _lib as L
    lib = L.load()
    g = np.random.default_rng(40 + ctas)
    for m in (1050, 300):
        A = g.standard_normal((m, m + 3)) / np.sqrt(m)
        H = A @ A.T + 0.3 * np.eye(m)
        b = g.standard_normal(m)
        ref = sp.spsvm_solve_mixed(_t(H), _t(b))
        lib.spsvm_set_factor_ctas(ctas)
        try:
            info, st, x, iters, be = sp.spsvm_solve_mixed(_t(H), _t(b))
            Hb = H.copy()
            Hb[m - 10, m - 10] = -5.0
            info_b, st_b, _, _, _ = sp.spsvm_solve_mixed(_t(Hb), _t(b))
        finally:
            lib.spsvm_set_factor_ctas(0)
        assert ref[0] == 0 and ref[1] == 0
        assert info == 0 and st == 0, (info, st, iters, be)
        xs, xr = x.cpu().numpy(), ref[2].cpu().numpy()
        assert np.max(np.abs(xs - xr)) <= 1e-9 * np.max(np.abs(xr))
        r = b - H @ xs
        assert np.max(np.abs(r)) <= 1e-13 * (np.max(np.abs(H).sum(1)) * np.max(np.abs(xs)) + np.max(np.abs(b)))
        # the FP32 factor breaks down at the planted pivot or before it
        assert 1 <= info_b <= m - 9 and st_b is None, (info_b, st_b)
        code = ctypes.c_int32()
        assert lib.spsvm_device_status(ctypes.byref(code)) == 0, code.value
