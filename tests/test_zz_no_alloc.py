"""The allocation-free CFL entry point against the context-based one.

aeth_cfl_dt_noalloc serves callers that may not allocate device memory
(for example code that runs inside another framework's caching allocator or
a host callback): it keeps its reduction scratch in a static device array.
This test calls it through the C ABI on a caller-owned FP64 state and
checks it against aeth_compute_dt on the same state, twice in a row (the
second call reuses the scratch the first one left behind).  The file name
makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _device_state(st, torch):
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (st.cons, st.b1, st.b2, st.b3)]
    return t


def test_noalloc_cfl_matches_context_dt_twice():
    import torch
    stream = torch.cuda.current_stream()
    for seed, n in ((51, (20, 18, 13)), (52, (33, 7, 9))):
        st = I.smooth_random_mhd(I.Block(n), seed, v_rms=0.8, b_rms=0.6, B0=(0.3, -0.2, 0.1))
        sv = A.Solver(A.make_config(precision=A.FP64), [A.make_block(n)], stream=stream)
        try:
            sv.set_state(0, st.cons, st.b1, st.b2, st.b3)
            dt_ref = sv.compute_dt()
        finally:
            sv.close()
        dev = _device_state(st, torch)
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        dx = [1.0 / n[0], 1.0 / n[1], 1.0 / n[2]]
        mem = []
        for call in range(2):
            torch.cuda.synchronize()
            mem.append((torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]))
            A.aeth_cfl_dt_noalloc(dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(),
                                  dev[3].data_ptr(), n, dx, 5.0 / 3.0, 1e-12, 1e-10, 0.3, True,
                                  out[call].data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        mem.append((torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]))
        # the second call allocates nothing: neither torch's allocator nor
        # the device's free memory moves across it (the first call may load
        # the library's device code, and with it the static scratch)
        assert mem[2] == mem[1], mem
        got = out.cpu().numpy()
        assert np.all(np.abs(got - dt_ref) <= 1e-14 * dt_ref), (got, dt_ref)


def test_noalloc_rejects_oversize_and_flags_nonfinite():
    import torch
    stream = torch.cuda.current_stream()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AethError):
        # ny * nz beyond the static scratch (2^18 rows)
        A.aeth_cfl_dt_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                              dummy.data_ptr(), (4, 1024, 1024), (1, 1, 1), 5 / 3, 1e-12, 1e-10,
                              0.3, True, dummy.data_ptr(), stream.cuda_stream)
    n = (8, 8, 8)
    cons = np.ones((5,) + n[::-1]); cons[1:4] = 0.0; cons[4] = 2.0
    cons[0, 2, 3, 4] = np.nan
    c = torch.from_numpy(cons).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    A.aeth_cfl_dt_noalloc(c.data_ptr(), 0, 0, 0, n, (0.125,) * 3, 5 / 3, 1e-12, 1e-10, 0.3, False,
                          out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
