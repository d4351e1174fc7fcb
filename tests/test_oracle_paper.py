"""Pins of the paper-parameterisation oracle (oracle/paper.py): the cosine / temperature
decode of Eq. (dict_recon) against the free-key oracle through the exact rewrite, its
invariances and special cases, and central finite differences of every gradient."""
import numpy as np
import pytest

import oracle
from oracle import paper


def _case(seed, n=40, ds=16, df=48, M=12, mask_drop=0.2):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, ds))
    W = rng.normal(size=(ds, df)) / np.sqrt(ds)
    D = rng.normal(size=(M, df))
    D0 = D + rng.normal(size=D.shape) * 0.08 * (np.arange(M) % 2)[:, None]  # half the atoms past the radius
    F = rng.normal(size=(n, df))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    mask = (rng.uniform(size=n) >= mask_drop).astype(np.uint8)
    return Q, W, D, D0, F, mask


@pytest.mark.parametrize("tau", [0.05, 0.1, 1.0])
def test_cosine_form_equals_free_key_form(tau):
    Q, W, D, D0, F, mask = _case(1)
    U, C, A, Fh = paper.decode_paper(Q, W, D, tau)
    Qp, K, V, c = paper.free_key_form(Q, W, D, tau)
    S2, A2, Fh2 = oracle.decode(Qp, K, V, c)
    np.testing.assert_allclose(A2, A, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(Fh2, Fh, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(S2, C / tau, rtol=1e-11, atol=1e-12)
    # the loss of the two forms (C oracle vs numpy) agrees too
    cfg = oracle.LossConfig()
    po, _ = oracle.loss(Fh2, F, mask, D, D0, cfg, Q.shape[1])
    pp = paper.loss_paper(Fh, F, mask, D, D0, cfg)
    for k in ("cos", "l2", "tr", "total"):
        assert pp[k] == pytest.approx(po[k], rel=1e-11, abs=1e-14), k


def test_cosine_bounds_and_softmax_rows():
    Q, W, D, *_ = _case(2)
    _, C, A, _ = paper.decode_paper(Q, W, D, 0.1)
    assert np.all(np.abs(C) <= 1 + 1e-12)
    np.testing.assert_allclose(A.sum(1), 1.0, atol=1e-14)


def test_invariances():
    """Cosine similarity ignores the scale of u_p and of D_j: positive row scalings of Q and a
    positive scaling of W leave Fhat unchanged; scaling D scales Fhat (Fhat = A D)."""
    Q, W, D, *_ = _case(3)
    Fh = paper.decode_paper(Q, W, D, 0.2)[3]
    s = np.random.default_rng(0).uniform(0.1, 5.0, size=(Q.shape[0], 1))
    np.testing.assert_allclose(paper.decode_paper(Q * s, W, D, 0.2)[3], Fh, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(paper.decode_paper(Q, 3.7 * W, D, 0.2)[3], Fh, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(paper.decode_paper(Q, W, 2.5 * D, 0.2)[3], 2.5 * Fh, rtol=1e-12, atol=1e-13)


def test_special_cases():
    Q, W, D, *_ = _case(4)
    # one atom: every pixel decodes to it
    np.testing.assert_allclose(paper.decode_paper(Q, W, D[:1], 0.1)[3], np.repeat(D[:1], Q.shape[0], 0), rtol=1e-14)
    # very high temperature: uniform attention, Fhat = mean atom
    np.testing.assert_allclose(paper.decode_paper(Q, W, D, 1e9)[3], np.repeat(D.mean(0, keepdims=True), Q.shape[0], 0),
                               rtol=1e-7, atol=1e-9)
    # an atom parallel to u_p at low temperature takes all the weight
    U = Q @ W
    D2 = np.vstack([3.0 * U[0], D[1:]])
    A = paper.decode_paper(Q[:1], W, D2, 1e-3)[2]
    assert A[0, 0] > 1 - 1e-12


def _total(Q, W, D, D0, F, mask, tau, cfg):
    return paper.loss_paper(paper.decode_paper(Q, W, D, tau)[3], F, mask, D, D0, cfg)["total"]


@pytest.mark.parametrize("tau", [0.05, 0.1, 1.0])
def test_gradients_finite_differences(tau):
    Q, W, D, D0, F, mask = _case(5)
    cfg = oracle.LossConfig()
    dQ, dW, dD = paper.backward_paper(Q, W, D, D0, F, mask, cfg, tau)
    rng = np.random.default_rng(7)
    for name, X, G in (("Q", Q, dQ), ("W", W, dW), ("D", D, dD)):
        idx = [tuple(rng.integers(0, s) for s in X.shape) for _ in range(12)]
        for ix in idx:
            h = 1e-6 * max(1.0, abs(X[ix]))
            Xp, Xm = X.copy(), X.copy()
            Xp[ix] += h
            Xm[ix] -= h
            args_p = dict(Q=Q, W=W, D=D)
            args_m = dict(Q=Q, W=W, D=D)
            args_p[name], args_m[name] = Xp, Xm
            if name == "D":  # keep away from the trust-region kink
                for Dx in (Xp, Xm):
                    r = np.linalg.norm(Dx - D0, axis=1)
                    assert np.all(np.abs(r - cfg.delta) > 10 * h)
            fd = (_total(args_p["Q"], args_p["W"], args_p["D"], D0, F, mask, tau, cfg)
                  - _total(args_m["Q"], args_m["W"], args_m["D"], D0, F, mask, tau, cfg)) / (2 * h)
            assert G[ix] == pytest.approx(fd, rel=2e-5, abs=1e-9), (name, ix)


def test_rewrite_chain_rule():
    """The gradients reached through the free-key form (the C oracle's dQ', dK, dV chained
    back through q'_p = q_p / |q_p W| and k_j = W D_j^T / |D_j|) equal the direct-form
    gradients: the algebra of the rewrite, checked once in float64."""
    Q, W, D, D0, F, mask = _case(6)
    tau = 0.1
    cfg = oracle.LossConfig()
    dQ, dW, dD = paper.backward_paper(Q, W, D, D0, F, mask, cfg, tau)
    Qp, K, V, c = paper.free_key_form(Q, W, D, tau)
    cfg_c = oracle.LossConfig(logit_scale=c)
    _, A, Fh = oracle.decode(Qp, K, V, c)
    dQp, dK, dV = oracle.backward(Qp, K, V, D0, A, Fh, F, mask, cfg_c)
    G = W @ W.T
    r = 1.0 / np.linalg.norm(Q @ W, axis=1)
    s = (Q * dQp).sum(1)
    dQ2 = r[:, None] * (dQp - (r ** 2 * s)[:, None] * (Q @ G))
    Cm = (Q * (s * r ** 3)[:, None]).T @ Q
    nd = np.linalg.norm(D, axis=1)
    g = dK @ W
    dW2 = dK.T @ (D / nd[:, None]) - Cm @ W
    dD2 = dV + (g - ((D * g).sum(1) / nd ** 2)[:, None] * D) / nd[:, None]
    np.testing.assert_allclose(dQ2, dQ, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dW2, dW, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dD2, dD, rtol=1e-9, atol=1e-12)
