"""The allocation-free min_eig entry point (psdproj_min_eig_noalloc).

Some callers cannot call cudaMalloc (a host library's memory manager owns the
device memory, or allocations are forbidden in its hot path).  For them the
library offers min_eig with its scratch in a fixed device array instead of a
context workspace.  This test calls it through the C ABI, twice in a row (the
second call must not see stale scratch), and compares it with the regular
psdproj_min_eig entry point on the same matrix, within the tolerance the
other min_eig tests use; it checks that the calls allocate no device memory,
that an oversized problem is rejected before anything runs, and that a host
pointer is refused.  This file is named to be collected last.
"""
import ctypes
import gc

import numpy as np
import pytest

import synth_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2410_19208_gb300 as ps  # noqa: E402


def _noalloc(A, N, seed, stream, out):
    n = A.shape[0]
    base = out.data_ptr()
    return ps.lib().psdproj_min_eig_noalloc(
        ctypes.c_void_p(A.data_ptr()), n, A.stride(0), N, seed, ctypes.c_void_p(base),
        ctypes.c_void_p(base + 8), ctypes.c_void_p(base + 16), ctypes.c_void_p(stream.cuda_stream))


# n = 4096 (a multiple of the product's 128-column tiles, 16-byte aligned A)
# takes the unmasked vector path; the others the masked one
@pytest.mark.parametrize("n,seed", [(2051, 3), (777, 5), (4096, 7)])
def test_noalloc_min_eig_matches_regular_entry_point(n, seed):
    Vr, lam = si.make_problem("small", n)
    A = torch.from_numpy(si.form_A_numpy(Vr, lam).astype(np.float32)).cuda()
    assert A.data_ptr() % 16 == 0
    stream = torch.cuda.current_stream()
    ctx = ps.Context(0, stream)
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.min_eig(A, 10, seed, alpha, s1, s2)
    assert ctx.sync_status() == 0
    ref = np.array([alpha.item(), s1.item(), s2.item()])
    ctx.close()
    tol = 1e-5 * (ref[1] + ref[2])
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for i in range(2):  # two calls in a row share the same scratch
        if i == 1:
            # nothing is allocated by the call: the device's free memory and
            # torch's allocator are unchanged across it (earlier tests'
            # cyclic garbage collected first, the collector held off while
            # measuring, so that no tensor is freed in between)
            gc.collect()
            gc.disable()
        try:
            free0, _ = torch.cuda.mem_get_info()
            alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
            code = _noalloc(A, 10, seed, stream, out)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            alloc1, reserved1 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        finally:
            gc.enable()
        assert code == 0, ps.STATUS.get(code)
        if i == 1:
            assert free1 == free0
            assert alloc1 == alloc0 and reserved1 == reserved0
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= tol), (got, ref)


def test_noalloc_rejects_sizes_above_its_scratch_and_host_memory():
    limit = 131072
    A = torch.zeros(1, 1, device="cuda")
    code = ps.lib().psdproj_min_eig_noalloc(ctypes.c_void_p(A.data_ptr()), limit + 1, limit + 1,
                                           10, 1, ctypes.c_void_p(A.data_ptr()), None, None, None)
    assert code == 8  # PSDPROJ_ETOOLARGE, returned before any launch
    Ah = torch.zeros(8, 8)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    code = ps.lib().psdproj_min_eig_noalloc(ctypes.c_void_p(Ah.data_ptr()), 8, 8, 10, 1,
                                           ctypes.c_void_p(out.data_ptr()), None, None, None)
    assert code == 1  # PSDPROJ_EINVAL: A is not device memory of the current device
