"""render_forward_static: forward path tracing for callers that cannot
allocate device memory (an application whose allocator owns all device
memory, or code running where allocation is forbidden after start-up).

The entry point keeps the scene tables in a fixed device array inside the
library instead of a pt_scene.  Its images must equal render_forward's on
the same inputs, call after call (the array is rewritten each time).  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2110_00085_gb300 import native as N
from paper_2110_00085_gb300 import synth

from _parity import RTOL, assert_images_close, t32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def test_static_entry_matches_scene_entry_on_two_calls():
    rng = np.random.default_rng(17)
    # call 1: the 32^3 blob scene, 9 cameras of 32x32
    sc1 = synth.config(1, n_paths=1 << 14)
    # call 2: a different grid, camera set and extinction (air, two types),
    # so stale tables from call 1 would show
    sc2 = synth.config(2, n_paths=1 << 12)
    sc2 = sc2.replace(cameras=synth.arc_cameras(5, sc2.box_size, 48, 40))
    for sc, seed in ((sc1, 11), (sc2, 12)):
        beta = (sc.beta_cloud * rng.uniform(0.9, 1.1, size=sc.beta_cloud.shape)).astype(np.float32)
        b = t32(beta)
        got = N.render_forward_static(sc, b, sc.n_paths, seed)
        ref = N.Scene(sc).render_forward(b, sc.n_paths, seed)
        torch.cuda.synchronize()
        assert ref.abs().max().item() > 0
        assert_images_close(got.cpu().numpy(), ref.cpu().numpy(), rtol=RTOL, what="static entry images")


def test_static_entry_allocates_no_device_memory():
    """The property the entry point exists for: after the first call on the
    device (which looks up the array's address and loads the kernel),
    repeated calls into a caller-owned image buffer leave the device's free
    memory and torch's reserved memory unchanged."""
    sc = synth.config(1, n_paths=1 << 12)
    b = t32(sc.beta_cloud)
    img = torch.zeros(sc.n_pixels, dtype=torch.float64, device=b.device)
    first = N.render_forward_static(sc, b, sc.n_paths, 3, images=img)
    assert first.data_ptr() == img.data_ptr()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for k in range(5):
        N.render_forward_static(sc, b, sc.n_paths, 4 + k, images=img)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert img.abs().max().item() > 0


def test_static_entry_rejects_scenes_over_its_limits():
    sc = synth.config(1, n_paths=16)
    b = t32(sc.beta_cloud)
    big = sc.replace(cameras=synth.arc_cameras(17, sc.box_size, 8, 8))
    with pytest.raises(RuntimeError, match="at most 16"):
        N.render_forward_static(big, b, 16, 1)
    wide = sc.replace(cameras=synth.arc_cameras(1, sc.box_size, 1024, 512))
    with pytest.raises(RuntimeError, match="pixels"):
        N.render_forward_static(wide, b, 16, 1)
