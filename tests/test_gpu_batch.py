"""The batched step (latentam_step_batch): several keyframes of one room sharing the
dictionary and the map's queries, against the oracle's pooled batch iteration."""
import numpy as np
import pytest

import oracle
from workloads import room_views

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def views():
    return room_views(3, n_views=3, n=40_000, width=96, height=72, fx=78.75)


def _adam_first(x0, g, lr=0.01):
    x = x0.astype(np.float64).copy()
    m, v = np.zeros_like(x), np.zeros_like(x)
    oracle.adam(x.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), 1, lr)
    return x


def test_batch_step_matches_oracle(api, ctx, views):
    st = api.LatentBatchStep(ctx, views, precision=api.FP32)
    assert len(st.queries) == 1  # the views share the map's queries
    loss = st.step(iters=1, learn_f=True)
    o = oracle.iteration_batch(views, oracle.LossConfig())
    assert loss["total"] == pytest.approx(o["loss"]["total"], rel=1e-4)
    assert loss["n_valid"] == o["loss"]["n_valid"]
    lr = 0.01
    for name, dev_t, x0, g in (("f", st.queries[0], views[0].f, o["df"][id(views[0].f)]),
                               ("K", st.K, views[0].K, o["dK"]), ("V", st.V, views[0].V, o["dV"])):
        want = _adam_first(x0, g, lr)
        got = dev_t.cpu().numpy().astype(np.float64)
        well = np.abs(g) > 1e-2 * np.abs(g).max()
        np.testing.assert_allclose(got[well], want[well], rtol=0, atol=1e-4 * lr + 1e-6, err_msg=name)


def test_batch_of_one_equals_single_step(api, ctx, views):
    a = api.LatentBatchStep(ctx, views[:1], precision=api.FP32)
    b = api.LatentStep(ctx, views[0], precision=api.FP32)
    la = a.step(iters=2, learn_f=True)
    lb = b.step(iters=2, learn_f=True)
    assert la["total"] == pytest.approx(lb["total"], rel=1e-6)
    torch.testing.assert_close(a.V, b.V, rtol=1e-6, atol=1e-7)
    torch.testing.assert_close(a.queries[0], b.f, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_stage2_keeps_queries(api, ctx, views, prec):
    p = api.FP32 if prec == "fp32" else api.BF16
    st = api.LatentBatchStep(ctx, views, precision=p,
                             target_dtype=torch.float32 if prec == "fp32" else torch.bfloat16)
    f0, V0 = st.queries[0].clone(), st.V.clone()
    l0 = st.step(iters=1, learn_f=False)
    l1 = st.step(iters=3, learn_f=False)
    assert torch.equal(st.queries[0], f0)
    assert np.isfinite(l0["total"]) and np.isfinite(l1["total"])
    assert st.adam_cfg.step == 5
    # four Adam steps of lr 0.01 move every value entry by at most 0.04
    moved = (st.V - V0).abs()
    assert float(moved.max()) <= 0.04 + 1e-5 and float(moved.mean()) > 1e-3


def test_uneven_keyframes_own_maps_shared_dictionary(api, ctx):
    """Keyframes of three resolutions, each with its own map and queries, one dictionary of
    M = 512 atoms of D = 768 (the batched workload's shapes, scaled down)."""
    from workloads import keyframe_batch
    frames = keyframe_batch(7, sizes=((48, 36), (96, 72), (80, 60)), ns=(15_000, 40_000, 25_000))
    st = api.LatentBatchStep(ctx, frames, precision=api.FP32)
    assert len(st.queries) == 3
    loss = st.step(iters=1, learn_f=True)
    o = oracle.iteration_batch(frames, oracle.LossConfig())
    assert loss["total"] == pytest.approx(o["loss"]["total"], rel=1e-4)
    assert loss["n_valid"] == o["loss"]["n_valid"]
    lr = 0.01
    checks = [("K", st.K, frames[0].K, o["dK"]), ("V", st.V, frames[0].V, o["dV"])]
    checks += [(f"f{k}", st.queries[k], frames[k].f, o["df"][id(frames[k].f)]) for k in range(3)]
    for name, dev_t, x0, g in checks:
        want = _adam_first(x0, g, lr)
        got = dev_t.cpu().numpy().astype(np.float64)
        well = np.abs(g) > 1e-2 * np.abs(g).max()
        np.testing.assert_allclose(got[well], want[well], rtol=0, atol=1e-4 * lr + 1e-6, err_msg=name)
    # the tensor-core form of the same batch
    st16 = api.LatentBatchStep(ctx, frames, precision=api.BF16, target_dtype=torch.bfloat16)
    l16 = st16.step(iters=1, learn_f=True)
    assert l16["total"] == pytest.approx(o["loss"]["total"], rel=5e-3)


def test_large_dictionary_ten_iterations(api, ctx):
    """A keyframe with M = 1024 atoms of D = 768 (the large-map workload's dictionary) run for
    ten Stage-I iterations: the first against the oracle, all finite."""
    from workloads import room_scene
    s = room_scene(8, n=60_000, d=32, M=1024, D=768, width=96, height=72, fx=78.75)
    o = oracle.iteration(s, oracle.LossConfig())
    for prec, tdt, rel in ((api.FP32, torch.float32, 1e-4), (api.BF16, torch.bfloat16, 5e-3)):
        st = api.LatentStep(ctx, s, precision=prec, target_dtype=tdt)
        l0 = st.step(iters=1)
        assert l0["total"] == pytest.approx(o["loss"]["total"], rel=rel)
        l9 = st.step(iters=9)
        assert np.isfinite(l9["total"]) and st.adam_cfg.step == 11
