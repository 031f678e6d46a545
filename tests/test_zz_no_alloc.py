"""hsma_coulomb_sum_static: the direct Coulomb sum for callers that cannot
allocate device memory during a call (a host whose memory manager owns the
device, a loop that cannot afford cudaFree's device-wide synchronisation).
It works in a fixed static device array inside the library.  Checked through
the C ABI against the allocating entry point hsma_coulomb_sum, on two calls
in a row whose sizes differ, so stale contents of the shared array would
show.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-6}  # relative RMS, as in the coulomb_sum parity test


def _inputs(ns, nt, seed):
    g = np.random.default_rng(seed)
    src = np.concatenate([g.random((ns, 3)) * 2 - 1, g.standard_normal((ns, 1))], axis=1)
    tgt = g.random((nt, 3)) * 2 - 1
    tgt[: nt // 4] = src[: nt // 4, :3]  # targets on sources: those pairs are skipped
    return src, tgt


def _abi_call(name, src, tgt, prec):
    import torch
    from paper_1806_04801_gb300 import hsma
    ds = torch.as_tensor(src).cuda()
    dt = torch.as_tensor(tgt).cuda()
    pot = torch.full((tgt.shape[0],), np.nan, dtype=torch.float64, device="cuda")
    fld = torch.full((tgt.shape[0], 3), np.nan, dtype=torch.float64, device="cuda")
    fn = getattr(hsma.lib(), name)
    rc = fn(ctypes.c_int64(src.shape[0]), ctypes.c_void_p(ds.data_ptr()), ctypes.c_int64(tgt.shape[0]),
            ctypes.c_void_p(dt.data_ptr()), ctypes.c_void_p(pot.data_ptr()), ctypes.c_void_p(fld.data_ptr()),
            ctypes.c_int(prec), None)
    torch.cuda.synchronize()
    return rc, pot.cpu().numpy(), fld.cpu().numpy()


def _rms(a):
    return float(np.sqrt(np.mean(np.asarray(a) ** 2)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    from paper_1806_04801_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", [1, 0])
def test_static_entry_point_matches_allocating_one_twice(prec):
    from paper_1806_04801_gb300 import hsma
    for call, (ns, nt, seed) in enumerate([(60000, 4000, 11), (7001, 1333, 12)]):
        src, tgt = _inputs(ns, nt, seed + 10 * prec)
        allocs_before = hsma.allocation_calls()
        rc, pot, fld = _abi_call("hsma_coulomb_sum_static", src, tgt, prec)
        assert rc == 0, f"call {call}: code {rc}"
        # the library made no allocation or free call during this call
        assert hsma.allocation_calls() == allocs_before
        rc2, pot_ref, fld_ref = _abi_call("hsma_coulomb_sum", src, tgt, prec)
        assert rc2 == 0
        assert hsma.allocation_calls() > allocs_before  # the counter sees the allocating entry point's calls
        assert np.all(np.isfinite(pot)) and np.all(np.isfinite(fld))
        assert _rms(pot - pot_ref) <= TOL[prec] * _rms(pot_ref), (call, _rms(pot - pot_ref) / _rms(pot_ref))
        assert _rms(fld - fld_ref) <= 10 * TOL[prec] * _rms(fld_ref)


def test_static_entry_point_rejects_calls_beyond_its_array():
    from paper_1806_04801_gb300 import hsma
    src, tgt = _inputs(1_200_000, 100, 5)  # 38 MB of source records > 32 MiB
    allocs_before = hsma.allocation_calls()
    rc, pot, _ = _abi_call("hsma_coulomb_sum_static", src, tgt, 1)
    assert rc == -11 and "memory budget" in hsma.strerror(rc)
    assert hsma.allocation_calls() == allocs_before
    assert np.all(np.isnan(pot))  # no work was done
