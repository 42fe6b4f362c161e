"""The entry point that allocates no device memory: afe_conserved_totals_noalloc.

It exists for callers that may not call cudaMalloc where they need the result (code
inside a framework whose caching allocator owns the device memory, or a loop that must
stay free of allocation and of the device synchronisation cudaMalloc/cudaFree imply).
Its partial sums live in a fixed device array inside the library instead of allocated
scratch.  This test calls it through the C ABI twice in a row, on two different states,
and checks each result against the totals from the existing entry point afe_get_stats.
The file sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_totals_match_afe_get_stats_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from inputs import states
    from inputs.voronoi import periodic_voronoi
    from paper_2605_00619_gb300 import afe

    pm = periodic_voronoi(8)
    p = afe.afe_default_params(3)
    h = afe.create_from_polymesh(pm, p)
    try:
        n = afe.afe_num_nodes(h)
        assert n > afe.AFE_NOALLOC_CHUNK          # several partial sums are combined
        x = afe.afe_get_node_coords(h)
        out = torch.empty(5, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        for u in (states.density_wave(x), states.constant(x, rho=1.3, vel=(0.1, 0.2, -0.3), p=0.7)):
            afe.afe_set_state(h, u)
            expected = np.array(afe.afe_get_stats(h).totals)
            dq = torch.from_numpy(u).to("cuda")
            out.fill_(float("nan"))
            afe.afe_conserved_totals_noalloc(h, dq.data_ptr(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), expected, rtol=1e-13, atol=0)
    finally:
        afe.afe_mesh_destroy(h)


_FIRST_CALL_IN_CAPTURE = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
from inputs import states
from inputs.voronoi import periodic_voronoi
from paper_2605_00619_gb300 import afe
pm = periodic_voronoi(2)
h = afe.create_from_polymesh(pm, afe.afe_default_params(1))
u = states.density_wave(afe.afe_get_node_coords(h))
afe.afe_set_state(h, u)
dq = torch.from_numpy(u).to("cuda")
out = torch.zeros(5, dtype=torch.float64, device="cuda")
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    out.add_(1.0)
    st = afe.afe_conserved_totals_noalloc(h, dq.data_ptr(), out.data_ptr(), s.cuda_stream, check=False)
    msg = afe.afe_last_error()
torch.cuda.synchronize()
st2 = afe.afe_conserved_totals_noalloc(h, dq.data_ptr(), out.data_ptr(), 0, check=False)
torch.cuda.synchronize()
ok = np.allclose(out.cpu().numpy(), np.array(afe.afe_get_stats(h).totals), rtol=1e-13, atol=0)
afe.afe_mesh_destroy(h)
print("RESULT", st, st2, int(ok), "capture" in msg)
"""


def test_first_call_inside_a_stream_capture_is_refused():
    """In a fresh process, the first call on the device made while a stream is being captured
    returns AFE_EINVAL without touching the device (it would have to look up the scratch
    array's address inside the capture); the next call, after the capture, works."""
    import os
    import subprocess
    import sys

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_IN_CAPTURE.format(root=root)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1].split()
    from paper_2605_00619_gb300 import afe
    assert int(line[1]) == afe.AFE_EINVAL and line[4] == "True"
    assert int(line[2]) == afe.AFE_OK and line[3] == "1"
