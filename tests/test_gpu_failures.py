"""The failure paths of the bounded device waits and of non-finite values, made to happen on
purpose without any GPU fault: a look-back wait of the radix sort pointed at a word that
nothing writes (with a short limit), the flag a tensor-core kernel raises when one of its
waits gives up, and a non-finite target.  Each must come back as a status from the next
synchronising call, and the context must stay usable: the next binning equals a clean one."""
import numpy as np
import pytest

from workloads import random_scene, room_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def scene():
    # about 20k pairs: twenty 1024-key blocks per radix pass, so a block has a predecessor
    return room_scene(1, n=300_000).crop(240, 180, 160, 120)


def _bins(api, ctx, s):
    proj = api.project(ctx, s.means, s.quats, s.scales, s.opacities, s.camera)
    return proj, api.sort(ctx, proj, s.camera)


def test_lookback_wait_gives_up_and_reports_timeout(api, scene):
    from paper_2602_12314_gb300 import _lib as L
    with api.Context(0) as ctx:
        proj, ref = _bins(api, ctx, scene)
        assert ref.num_pairs > 2048
        want_pairs = ref.pair_ids[:ref.num_pairs].clone()
        want_ranges = ref.tile_ranges.clone()
        ctx.test_wait_timeout(0)
        armed = api.sort(ctx, proj, scene.camera)  # its look-back gives up: tiles left empty
        torch.cuda.synchronize()
        assert int(armed.tile_ranges.abs().sum()) == 0
        with pytest.raises(L.LatentamError) as e:
            api.sort(ctx, proj, scene.camera)
        assert e.value.status == L.ERR_TIMEOUT and "look-back" in str(e.value)
        again = api.sort(ctx, proj, scene.camera)  # reported and cleared: a clean binning
        assert again.num_pairs == ref.num_pairs
        assert torch.equal(again.pair_ids[:again.num_pairs], want_pairs)
        assert torch.equal(again.tile_ranges, want_ranges)


def test_tensor_core_wait_flag_reported_once(api, scene):
    from paper_2602_12314_gb300 import _lib as L
    s = random_scene(5, n=2000, d=32, M=64, D=256, width=48, height=40, log_scale=-2.6)
    with api.Context(0) as ctx:
        proj, _ = _bins(api, ctx, s)
        ctx.test_wait_timeout(1)
        with pytest.raises(L.LatentamError) as e:
            api.sort(ctx, proj, s.camera)
        assert e.value.status == L.ERR_TIMEOUT and "tensor-core" in str(e.value)
        api.sort(ctx, proj, s.camera)  # cleared
        st = api.LatentStep(ctx, s, precision=api.BF16)
        ctx.test_wait_timeout(1)
        with pytest.raises(L.LatentamError) as e:
            st.step(iters=1)
        assert e.value.status == L.ERR_TIMEOUT
        loss = st.step(iters=1)
        assert np.isfinite(loss["total"])


def test_non_finite_loss_reported(api):
    from paper_2602_12314_gb300 import _lib as L
    s = random_scene(6, n=2000, d=32, M=64, D=256, width=48, height=40, log_scale=-2.6)
    s.F[5, :] = np.nan
    with api.Context(0) as ctx:
        st = api.LatentStep(ctx, s, precision=api.FP32)
        with pytest.raises(L.LatentamError) as e:
            st.step(iters=1)
        assert e.value.status == L.ERR_NOT_FINITE


def test_unknown_wait_rejected(api):
    from paper_2602_12314_gb300 import _lib as L
    with api.Context(0) as ctx:
        with pytest.raises(L.LatentamError) as e:
            ctx.test_wait_timeout(7)
        assert e.value.status == L.ERR_INVALID_ARG
