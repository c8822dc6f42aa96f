"""Bounded device waits: a wait that gives up reports SPSVM_ERR_TIMEOUT on
the stream its kernel ran on, leaves the context usable, and is invisible to
work on other streams.  The waits are made to give up by a short poll limit
(spsvm_set_wait_limit) on the triangular solves' flag and tag polls, whose
producers take microseconds: no fault, trap or unbounded wait is involved."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SPSVM_ERR_TIMEOUT = -6


@pytest.fixture(scope="module")
def sp():
    import paper_1404_1066_gb300 as sp
    sp.load()
    return sp


def _spd(m, seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, m + 8)) / np.sqrt(m)
    return A @ A.T + 0.5 * np.eye(m)


def test_short_wait_limit_times_out_and_recovers(sp):
    lib = sp.load()
    m = 4096
    H = torch.from_numpy(_spd(m, 1)).cuda()
    b = torch.randn(m, dtype=torch.float64, device="cuda")
    wb = lib.spsvm_mixed_work_bytes(m)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.zeros(m, dtype=torch.float64, device="cuda")
    assert lib.spsvm_cholesky_mixed(H.data_ptr(), m, m, 0.0, info.data_ptr(), work.data_ptr(), wb,
                                    None) == 0
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    try:
        lib.spsvm_set_wait_limit(1)
        rc = lib.spsvm_solve_mixed(H.data_ptr(), m, m, 0.0, b.data_ptr(), x.data_ptr(), 30, 1e-13,
                                   None, None, work.data_ptr(), wb, None)
    finally:
        lib.spsvm_set_wait_limit(0)
    assert rc == SPSVM_ERR_TIMEOUT
    # the solve read and cleared its stream's word; the context still works
    code = ctypes.c_int32(-9)
    assert lib.spsvm_device_status(ctypes.byref(code)) == 0 and code.value == 0
    rc = lib.spsvm_solve_mixed(H.data_ptr(), m, m, 0.0, b.data_ptr(), x.data_ptr(), 30, 1e-13,
                               None, None, work.data_ptr(), wb, None)
    assert rc == 0
    r = (b - H @ x).abs().max().item()
    assert r <= 1e-12 * (H.abs().sum(1).max().item() * x.abs().max().item() + b.abs().max().item())


def test_timeout_is_reported_on_its_own_stream(sp):
    """A FP64 solve whose waits give up on stream A records its site code in
    A's status word only: a healthy solve on stream B reports OK, then A
    reports TIMEOUT (and is clear after that read)."""
    lib = sp.load()
    m = 8192
    Hn = _spd(m, 2)
    Lf = torch.from_numpy(Hn.copy()).cuda()
    assert sp.spsvm_cholesky(Lf) == 0   # factor and diagonal-block inverses, in place
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    swb = lib.spsvm_cholesky_solve_work_bytes(m)
    wa = torch.empty(swb, dtype=torch.uint8, device="cuda")
    wbuf = torch.empty(swb, dtype=torch.uint8, device="cuda")
    ba = torch.randn(m, dtype=torch.float64, device="cuda")
    bb = torch.randn(m, dtype=torch.float64, device="cuda")
    bb_ref = bb.clone()
    torch.cuda.synchronize()
    try:
        lib.spsvm_set_wait_limit(1)
        assert lib.spsvm_cholesky_solve(Lf.data_ptr(), m, m, ba.data_ptr(), wa.data_ptr(), swb,
                                        ctypes.c_void_p(sa.cuda_stream)) == 0
    finally:
        lib.spsvm_set_wait_limit(0)
    sa.synchronize()
    assert lib.spsvm_cholesky_solve(Lf.data_ptr(), m, m, bb.data_ptr(), wbuf.data_ptr(), swb,
                                    ctypes.c_void_p(sb.cuda_stream)) == 0
    code = ctypes.c_int32(-9)
    assert lib.spsvm_stream_status(ctypes.c_void_p(sb.cuda_stream), ctypes.byref(code)) == 0
    assert code.value == 0
    x = bb.cpu().numpy()
    np.testing.assert_allclose(Hn @ x, bb_ref.cpu().numpy(), rtol=0, atol=1e-9 * np.abs(bb_ref.cpu().numpy()).max())
    assert lib.spsvm_stream_status(ctypes.c_void_p(sa.cuda_stream), ctypes.byref(code)) == SPSVM_ERR_TIMEOUT
    assert code.value in (221, 222)
    assert lib.spsvm_stream_status(ctypes.c_void_p(sa.cuda_stream), ctypes.byref(code)) == 0
    assert code.value == 0
