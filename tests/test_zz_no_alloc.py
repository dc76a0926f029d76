"""The allocation-free Green's-function entry point (vie_green_noalloc).

Callers that cannot allocate device memory while they run (a framework that
owns all of HBM through its own pool, or code that must not let an allocation
synchronise the device) pass their own device buffers; the entry point keeps
its interpolation tables in a static device array.  This test checks it
against the allocating entry point vie_green on two calls in a row with
different incidences, so that the second call cannot reuse the first call's
tables.  It lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import cellgen

pytestmark = pytest.mark.gpu

vie = pytest.importorskip("paper_1809_05334_gb300.vie")
torch = pytest.importorskip("torch")


def _points(a, b, zmax, n=300, seed=5):
    rng = np.random.default_rng(seed)
    d = np.stack([rng.uniform(-a, a, n) * 0.999, rng.uniform(-b, b, n) * 0.999, rng.uniform(-zmax, zmax, n)], 1)
    d[:5, 2] = 0.0
    return d


# FP64: the same series on both sides (relative 1e-12).  FP32: the entry
# without allocations evaluates the general tabulated form, the allocating
# entry the fill's short form (another summation order of the same tables);
# each is within 2e-6 max|g| of the FP64 oracle (the FP32 g_p bar of
# test_gpu_parity), so they agree to 4e-6 max|g|.
@pytest.mark.parametrize("precision,rtol,atol", [(0, 1e-12, 0.0), (1, 0.0, 4e-6)])
def test_green_noalloc_matches_allocating_entry(precision, rtol, atol):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    a, b, thick = 180.0, 150.0, 60.0
    cell = cellgen.slab_cell(2, 2, 1, a, b, thick, (2.0, 0.1))
    incidences = ((520.0, 0.0, 0.0), (430.0, 0.6, 0.3))
    s = vie.Solver(precision=vie.VIE_FP32)
    d = _points(a, b, thick)
    try:
        s.set_mesh(cell)
        refs = [s.green(d, lam, th, ph, precision) for lam, th, ph in incidences]
    finally:
        s.close()
    lib = vie.load()
    # the allocating entry covers |dz| up to max(mesh thickness, max|dz|)
    z_ext = max(thick, float(np.max(np.abs(d[:, 2]))))
    d_dev = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    out_dev = torch.zeros(2 * len(d), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def call(lam, th, ph):
        rc = lib.vie_green_noalloc(lam, th, ph, a, b, z_ext, ctypes.c_void_p(d_dev.data_ptr()),
                                   ctypes.c_void_p(out_dev.data_ptr()), len(d), precision,
                                   ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        return rc

    assert call(*incidences[1]) == 0          # first call: the one-time set-up on this device
    free0 = torch.cuda.mem_get_info()[0]
    for (lam, th, ph), ref in zip(incidences, refs):   # two calls in a row, different incidences
        out_dev.zero_()
        assert call(lam, th, ph) == 0
        got = out_dev.cpu().numpy().view(np.complex128)
        if rtol > 0:
            assert np.max(np.abs(got - ref) / np.abs(ref)) < rtol
        else:
            assert np.max(np.abs(got - ref)) < atol * np.max(np.abs(ref))
    # no device memory was taken by the calls
    assert torch.cuda.mem_get_info()[0] == free0


def test_green_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    lib = vie.load()
    d_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    out_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    assert lib.vie_green_noalloc(500.0, 0.0, 0.0, -1.0, 100.0, 10.0, p(d_dev.data_ptr()), p(out_dev.data_ptr()),
                                 1, 1, None) == -1
    assert lib.vie_green_noalloc(500.0, 0.0, 0.0, 100.0, 100.0, 10.0, p(d_dev.data_ptr()), p(out_dev.data_ptr()),
                                 1, 7, None) == -1
