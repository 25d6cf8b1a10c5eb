"""The roofline probes do the work they are credited with: the load probe
returns every thread's sum of the values it loaded (so the bytes counted
were delivered), and the reduction probe adds 1.0 per pass to exactly the
elements its lanes target and leaves the rest of the buffer alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import paper_2404_09531_gb300 as om  # noqa: E402


def test_load_probe_sums_every_loaded_value():
    ctas, per_cta, passes = 3, 16384, 5
    buf = torch.ones(ctas * per_cta // 4, device="cuda")
    sink = torch.full((ctas * 256,), -1.0, device="cuda")
    nbytes = om.probe_load_bandwidth(buf, per_cta, ctas, passes, sink)
    torch.cuda.synchronize()
    assert nbytes == ctas * per_cta * passes
    # a thread loads 8 floats every 256 x 8 floats of its CTA's slice
    want = 8.0 * (per_cta // 4) / 2048 * passes
    assert torch.all(sink == want)


def test_reduction_probe_adds_to_its_lines_only():
    ctas, per_warp, passes = 2, 8192, 3
    buf = torch.zeros(ctas * 8 * per_warp // 4 + 64, device="cuda")  # 64 guard floats after the regions
    nbytes = om.probe_red_bandwidth(buf, per_warp, ctas, passes)
    got = buf.cpu().numpy()
    assert nbytes == ctas * per_warp * passes
    want = np.zeros_like(got)
    fpw = per_warp // 4
    for w in range(ctas * 8):
        for step in range(fpw // 1024):
            for lane in range(32):
                o = w * fpw + step * 1024 + lane * 32
                want[o:o + 4] = passes
    assert np.array_equal(got, want)
    assert nbytes == 16 * 32 * (fpw // 1024) * ctas * 8 * passes  # 16 B per lane per step
