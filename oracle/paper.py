"""FP64 oracle of the paper's own parameterisation of the dictionary decode (Eq. dict_recon
with the cosine / temperature similarity of Sec. III-B).

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the product path).

The decode maps the rendered queries Q (n x d_s) through the projection W (d_s x d_f) to the
initial reconstructions U = Q W, compares each row of U with each atom of the dictionary
D (M x d_f) by cosine similarity after l2 normalisation, divides by the temperature tau, takes
the row softmax and mixes the atoms:

    C_pj = <u_p, D_j> / (max(|u_p|, 1e-12) max(|D_j|, 1e-12)),   A = softmax_rows(C / tau),
    Fhat = A D.

The loss is the feature objective of Eq. (feat_loss) (times lambda_f of Eq. full_obj) with the
trust region on the atoms D against D0 (the dictionary at the start of the keyframe).  Every
step below is written in this direct form, in numpy float64, in the order the paper states
it; the gradients follow the chain rule through the normalisations one factor at a time.

Parity status: pinned by tests/test_oracle_paper.py (the free-key oracle of
latentam_oracle.c under the exact rewrite k_j = W D_j^T / |D_j|, q'_p = q_p / |q_p W|,
c = 1/tau; invariances of the cosine form; central finite differences of dQ, dW, dD).
"""
from __future__ import annotations

import numpy as np

EPS_NORM = 1e-12  # floor of |u_p| and |D_j| in the normalisation
EPS_COS = 1e-8    # floor of |Fhat_p| |F_p| in the loss cosine (as in the free-key loss)


def _norms(X):
    return np.maximum(np.linalg.norm(X, axis=1), EPS_NORM)


def decode_paper(Q, W, D, tau: float):
    """Eq. (dict_recon) in the cosine / temperature form; returns (U, C, A, Fhat)."""
    Q, W, D = (np.asarray(x, np.float64) for x in (Q, W, D))
    U = Q @ W
    nu, nd = _norms(U), _norms(D)
    C = (U @ D.T) / nu[:, None] / nd[None, :]
    S = C / tau
    S = S - S.max(axis=1, keepdims=True)
    E = np.exp(S)
    A = E / E.sum(axis=1, keepdims=True)
    return U, C, A, A @ D


def loss_paper(Fhat, F, mask, D, D0, cfg):
    """lambda_f (lambda_cos mean_Omega(1 - cos_p) + lambda_2 mean_{Omega x d_f} |Fhat - F|^2
    + lambda_D sum_j relu(|D_j - D0_j| - delta)); returns the parts as a dict."""
    Fhat, F, D, D0 = (np.asarray(x, np.float64) for x in (Fhat, F, D, D0))
    m = np.asarray(mask).astype(bool)
    nv = int(m.sum())
    cos_p = (Fhat * F).sum(1) / np.maximum(np.linalg.norm(Fhat, axis=1) * np.linalg.norm(F, axis=1), EPS_COS)
    lcos = float((1.0 - cos_p[m]).sum() / nv) if nv else 0.0
    l2 = float(((Fhat[m] - F[m]) ** 2).sum() / (nv * F.shape[1])) if nv else 0.0
    tr = float(np.maximum(np.linalg.norm(D - D0, axis=1) - cfg.delta, 0.0).sum())
    total = cfg.lambda_f * (cfg.lambda_cos * lcos + cfg.lambda_2 * l2 + cfg.lambda_D * tr)
    return dict(cos=lcos, l2=l2, tr=tr, total=total, n_valid=nv)


def backward_paper(Q, W, D, D0, F, mask, cfg, tau: float):
    """Gradients of loss_paper(decode_paper(Q, W, D, tau)) with respect to Q, W and D."""
    Q, W, D, D0, F = (np.asarray(x, np.float64) for x in (Q, W, D, D0, F))
    U, C, A, Fh = decode_paper(Q, W, D, tau)
    m = np.asarray(mask).astype(bool)
    nv = int(m.sum())
    n, df = Fh.shape
    # dL/dFhat (loss-set rows only)
    dF = np.zeros_like(Fh)
    if nv:
        nh = np.linalg.norm(Fh, axis=1)
        nf = np.linalg.norm(F, axis=1)
        den = nh * nf
        dot = (Fh * F).sum(1)
        big = den > EPS_COS
        cos_p = dot / np.maximum(den, EPS_COS)
        # d(1 - cos_p)/dFhat_p
        g_cos = np.where(big[:, None],
                         -(F / np.maximum(den, EPS_COS)[:, None]) + (cos_p / np.maximum(nh, 1e-300) ** 2)[:, None] * Fh,
                         -F / EPS_COS)
        g_l2 = 2.0 * (Fh - F)
        dF = cfg.lambda_f * (cfg.lambda_cos * g_cos / nv + cfg.lambda_2 * g_l2 / (nv * df))
        dF[~m] = 0.0
    # Fhat = A D
    dA = dF @ D.T
    dD = A.T @ dF
    # A = softmax(C / tau)
    dS = A * (dA - (A * dA).sum(1, keepdims=True))
    dC = dS / tau
    # C_pj = <u_p, D_j> / (|u_p| |D_j|)
    nu, nd = _norms(U), _norms(D)
    Uh, Dh = U / nu[:, None], D / nd[:, None]
    dU = (dC @ Dh - (dC * C).sum(1, keepdims=True) * Uh) / nu[:, None]
    dD += (dC.T @ Uh - (dC * C).sum(0)[:, None] * Dh) / nd[:, None]
    # trust region on the atoms (subgradient 0 at the kink)
    dev = D - D0
    rn = np.linalg.norm(dev, axis=1)
    out = rn > cfg.delta
    dD[out] += cfg.lambda_f * cfg.lambda_D * dev[out] / rn[out, None]
    # U = Q W
    dQ = dU @ W.T
    dW = Q.T @ dU
    return dQ, dW, dD


def free_key_form(Q, W, D, tau: float):
    """The exact rewrite of the cosine form as the free-key decode: keys k_j = W D_j^T / |D_j|
    (M x d_s), values D, per-row query scale 1 / |q_p W| folded into the queries, logit scale
    1 / tau.  Returns (Q', K, V, c)."""
    Q, W, D = (np.asarray(x, np.float64) for x in (Q, W, D))
    K = (D @ W.T) / _norms(D)[:, None]
    Qp = Q / _norms(Q @ W)[:, None]
    return Qp, K, D, 1.0 / tau
