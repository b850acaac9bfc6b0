"""Gather roofline probes (measurement entry points): argument checks and
the ordering their access patterns imply."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_03095_b300 as mc  # noqa: E402


def test_mixed_probe_brackets_the_record_probe():
    foot = 64 << 20
    r64 = mc.mcmi_gather_roofline(foot, 128, 8, 32, record_bytes=64)
    r0 = mc.mcmi_gather_roofline_mix(foot, 16 << 20, 0.0, 128, 8, 32)
    r1 = mc.mcmi_gather_roofline_mix(foot, 16 << 20, 1.0, 128, 8, 32)
    rh = mc.mcmi_gather_roofline_mix(foot, 16 << 20, 0.5, 128, 8, 32)
    # no bucket reads: the same pattern as the 64-byte record probe
    assert 0.8 < r0 / r64 < 1.25, (r0, r64)
    # every record read followed by a dependent bucket read is slower, half of them in between
    assert r1 < rh < r0, (r1, rh, r0)


def test_mixed_probe_rejects_bad_arguments():
    with pytest.raises(mc.McmiError):
        mc.mcmi_gather_roofline_mix(1024, 1 << 20, 0.5)
    with pytest.raises(mc.McmiError):
        mc.mcmi_gather_roofline_mix(1 << 20, 1 << 20, 1.5)
    with pytest.raises(mc.McmiError):
        mc.mcmi_gather_roofline_mix(1 << 20, 1 << 20, 0.5, threads_per_block=2048)
