"""The allocation-free ready-set entry point (aw_ready_set_noalloc).

Some callers cannot allocate device memory: applications that own all device
memory through their own pool, or loops that must not pay cudaMalloc's
implicit device synchronisation.  For them the library offers one entry point
whose only scratch is a fixed device array.  This test calls it through the C
ABI, three times in a row on evolving states, and checks its output against what the
existing aw_lts_sweep entry point then does: the elements whose update count
grows in that sweep are exactly the listed ready set.  Between its second and
third call the device's free memory and torch's allocations must not move.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_ready_set_matches_the_sweep():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3719_gb300 import aleweno
    from paper_1408_3719_gb300 import workloads as W

    lib = aleweno.load()
    mesh, Q = W.explosion(0.02)
    s = aleweno.Solver(order_M=2, t_end=0.25)
    s.load_mesh(mesh)
    s.load_state(Q)
    n = mesh["tri"].shape[0]
    for _ in range(3):
        s.sweep()
    # the caller provides the outputs, allocated here before any call
    outs = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(3)]
    cnts = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in range(3)]
    for call in range(3):
        out, cnt = outs[call], cnts[call]
        torch.cuda.synchronize()  # the library runs on its own stream
        if call == 1:
            # the first call has loaded the kernels (lazy module loading
            # reserves device memory for code and for the fixed scratch);
            # from here on nothing may allocate device memory
            free0 = torch.cuda.mem_get_info()[0]
            torch0 = torch.cuda.memory_allocated()
        rc = lib.aw_ready_set_noalloc(s.h, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(cnt.data_ptr()))
        assert rc == 0, lib.aw_last_error(s.h)
        torch.cuda.synchronize()
        if call == 2:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == torch0
        k = int(cnt.item())
        listed = out[:k].cpu().numpy()
        assert k > 0
        assert np.all(np.diff(listed) > 0)  # ascending, no repeats
        assert np.all(out[k:].cpu().numpy() == -1)
        before, _ = s.update_counts()
        updated = s.sweep()
        after, _ = s.update_counts()
        assert updated == k, (call, updated, k)
        assert np.array_equal(np.nonzero(after - before)[0], listed)
