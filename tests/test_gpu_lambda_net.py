"""Learned lambda rule on the GPU: the network's forward, gradient and Adam kernels against the
FP64 oracle network, the training-data kernels (features of H_k, error-optimal labels) against
the oracle solve, the rule inside the hybrid step, and what the trained network gains over GCV.

Tolerances: FP32 mode 1e-5 relative (FP32 sums of at most 80 products against FP64); BF16
mode 1e-2 relative (operands rounded to 8 significant bits, relative error 2^-9 each, FP32
accumulation), as for any BF16 tensor-core layer.
"""
import math

import numpy as np
import pytest

import synth
from oracle import mlp as OM
from oracle import proj as OP
from oracle import solver as OS
from tests._common import gpu_geom, problem, rel, to_dev

pytestmark = pytest.mark.gpu

NP = 9569
B3 = 9408                   # offset of b3 in the parameter vector


KEYS = (("W1", (64, 80)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,)),
        ("b3", (1,)), ("mu", (80,)), ("isd", (80,)))


def _flat(p):
    return np.concatenate([p[k].ravel() for k, _ in KEYS])


def _unflat(v):
    v = np.asarray(v, np.float64)
    o = 0
    out = {}
    for key, shape in KEYS:
        size = int(np.prod(shape))
        out[key] = v[o:o + size].reshape(shape)
        o += size
    assert o == NP
    return out


def _params(seed, bias_scale=0.1):
    """Oracle-initialised weights, random biases and a non-trivial input standardisation."""
    p = OM.init_params(seed)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    for key in ("b1", "b2", "b3"):
        p[key] = bias_scale * rng.standard_normal(p[key].shape)
    p["mu"] = 0.3 * rng.standard_normal(80)
    p["isd"] = 0.5 + rng.random(80)
    v = np.asarray(_flat(p), np.float32)
    return v, _unflat(v.astype(np.float64))


def _bf16_case(p, X):
    """The BF16 network as the oracle sees it: weights rounded to BF16, biases FP32, and the
    input standardised in FP32 (as the kernel does) then rounded to BF16."""
    q = {k: OM.bf16_round(v) for k, v in p.items()}
    for key in ("b1", "b2", "b3"):
        q[key] = p[key]
    q["mu"] = np.zeros(80)
    q["isd"] = np.ones(80)
    Xs = (X.astype(np.float32) - p["mu"].astype(np.float32)) * p["isd"].astype(np.float32)
    return q, OM.bf16_round(Xs.astype(np.float64))


def _data(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.standard_normal((n, 80)).astype(np.float32)
    Y = rng.standard_normal(n).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("n", [1, 64, 150])
def test_forward_matches_oracle(bf16, n):
    import torch
    from paper_2602_17892_gb300._binding import ct_mlp_forward
    v, p = _params(1)
    X, _ = _data(n, 2)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ct_mlp_forward(to_dev(v), to_dev(X).reshape(n, 80), out, bf16=bf16)
    torch.cuda.synchronize()
    Xo = X.astype(np.float64)
    if bf16:
        ref, _ = OM.forward(*_bf16_case(p, X))
        assert rel(out.cpu().numpy(), ref) <= 1e-2
    else:
        ref, _ = OM.forward(p, Xo)
        assert rel(out.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_matches_oracle(bf16):
    """Every parameter block of the GPU gradient (150 rows: two full CTAs and a ragged one)
    against the oracle's analytic gradient, which central differences pin on the CPU."""
    import torch
    from paper_2602_17892_gb300._binding import ct_mlp_grad
    v, p = _params(3)
    n = 150
    X, Y = _data(n, 4)
    grad = torch.empty(NP, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ct_mlp_grad(to_dev(v), to_dev(X).reshape(n, 80), to_dev(Y), grad, loss, bf16=bf16)
    torch.cuda.synchronize()
    Xo, Yo = X.astype(np.float64), Y.astype(np.float64)
    pp, Xr = _bf16_case(p, X) if bf16 else (p, Xo)
    ref = OM.backward(pp, Xr, Yo)
    got = _unflat(grad.cpu().numpy())
    tol = 1e-2 if bf16 else 1e-5
    for key in ("W1", "b1", "W2", "b2", "w3", "b3"):
        assert rel(got[key], ref[key]) <= tol, (key, rel(got[key], ref[key]))
    assert not got["mu"].any() and not got["isd"].any()
    assert abs(float(loss.cpu()[0]) - OM.loss(pp, Xr, Yo)) <= tol * OM.loss(pp, Xr, Yo)


def test_gradient_is_deterministic_and_zero_at_a_fit():
    import torch
    from paper_2602_17892_gb300._binding import ct_mlp_forward, ct_mlp_grad
    v, _ = _params(5)
    X, _ = _data(200, 6)
    Xd = to_dev(X).reshape(200, 80)
    Pd = to_dev(v)
    Y = torch.empty(200, dtype=torch.float32, device="cuda")
    ct_mlp_forward(Pd, Xd, Y, bf16=True)          # targets = the network's own outputs
    g1 = torch.empty(NP, dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g1)
    ct_mlp_grad(Pd, Xd, Y, g1, bf16=True)
    ct_mlp_grad(Pd, Xd, Y, g2, bf16=True)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    assert float(g1.abs().max()) == 0.0


def test_adam_step_matches_oracle():
    import torch
    from paper_2602_17892_gb300._binding import ct_mlp_adam
    rng = np.random.Generator(np.random.PCG64(7))
    P = rng.standard_normal(NP).astype(np.float32)
    G = rng.standard_normal(NP).astype(np.float32)
    Mm = (0.1 * rng.standard_normal(NP)).astype(np.float32)
    V = np.abs(0.1 * rng.standard_normal(NP)).astype(np.float32)
    Pd, Gd, Md, Vd = (to_dev(a) for a in (P, G, Mm, V))
    ct_mlp_adam(Pd, Gd, Md, Vd, 3e-3, 5)
    torch.cuda.synchronize()
    p = {"w": P.astype(np.float64)}
    OM.adam_step(p, {"w": G.astype(np.float64)}, {"w": Mm.astype(np.float64)},
                 {"w": V.astype(np.float64)}, 5, lr=3e-3)
    assert rel(Pd.cpu().numpy() - P, p["w"] - P) <= 1e-4


def test_training_fits_a_teacher_network():
    """Targets from a random teacher network: the training kernels lower the loss by a factor
    of five, and two runs from the same start give identical parameters."""
    import torch
    from paper_2602_17892_gb300._binding import ct_mlp_forward, ct_mlp_train
    n = 4096
    X, _ = _data(n, 8)
    Xd = to_dev(X).reshape(n, 80)
    tv, _ = _params(9)
    Y = torch.empty(n, dtype=torch.float32, device="cuda")
    ct_mlp_forward(to_dev(tv), Xd, Y, bf16=True)
    v0, _ = _params(10)
    runs = []
    for _ in range(2):
        P = to_dev(v0)
        m = torch.zeros_like(P)
        vv = torch.zeros_like(P)
        lh = torch.empty(60 * 8, dtype=torch.float32, device="cuda")
        t = ct_mlp_train(P, m, vv, Xd, Y, 512, 60, 3e-3, loss_hist=lh)
        assert t == 60 * 8
        runs.append((P.clone(), lh.cpu().numpy()))
    assert torch.equal(runs[0][0], runs[1][0])
    lh = runs[0][1]
    assert lh[-8:].mean() < 0.2 * lh[:8].mean()


def _oracle_samples(g, b, x_true, K):
    A, B = OP.operators(g)
    ref = OS.hybrid_gmres("ab", A, B, b, K, rule="gcv")
    W = ref["W"]
    Z = np.stack([OP.back_pixel(g, W[j]).reshape(-1) for j in range(K)], axis=1)
    G, gv = Z.T @ Z, Z.T @ x_true
    H, beta = ref["H"], ref["beta"]
    feats, lams, errs = [], [], []
    for k in range(1, K + 1):
        Hk = H[:k + 1, :k]
        U, s, Vt = np.linalg.svd(Hk, full_matrices=True)
        feats.append(OM.features(k, K, s, beta * U[0, :], beta))
        lams.append(OM.optimal_lambda(Hk, beta, G[:k, :k], gv[:k]))
        errs.append(lambda lam, k=k, s=s, c=beta * U[0, :], Vt=Vt:
                    OM.tikhonov_error(lam, s, c, Vt, G[:k, :k], gv[:k]) + x_true @ x_true)
    return np.array(feats), np.array(lams), errs, H


@pytest.mark.parametrize("geom", [synth.parallel2d(48, 40, 71), synth.parallel2d(40, 30, 61, ny=28)])
def test_training_samples_match_oracle(geom):
    """ct_lambda_samples: features against the oracle's features of its own H_k, labels
    compared through the reconstruction error they give (the error's minimum is flat, so two
    correct searches may stop at slightly different lambda)."""
    import torch
    from paper_2602_17892_gb300._binding import ct_lambda_samples
    K = 12
    x_true, b, _ = problem(geom, 31, 0.02, 32)
    G = gpu_geom(geom)
    feats = torch.zeros((K, 80), dtype=torch.float32, device="cuda")
    labels = torch.zeros(K, dtype=torch.float32, device="cuda")
    x = torch.empty(G.n, dtype=torch.float32, device="cuda")
    xt = to_dev(x_true)
    info = ct_lambda_samples(G, to_dev(b), xt, x, feats, labels, max_iters=K, rule="gcv")
    assert info["iters_done"] == K
    Fo, lam_o, errs, _ = _oracle_samples(geom, b, xt.cpu().numpy().astype(np.float64), K)
    Fg = feats.cpu().numpy().astype(np.float64)
    Lg = labels.cpu().numpy().astype(np.float64)
    for k in range(1, K + 1):
        fo, fg = Fo[k - 1], Fg[k - 1]
        assert abs(fg[0] - fo[0]) < 1e-7
        big = fo[1:33] > -3.0                     # sigma_i / sigma_1 > 1e-3: well conditioned
        assert np.all(np.abs(fg[1:33][big] - fo[1:33][big]) < 1e-3), k
        assert np.all(np.abs(fg[33:65][big] - fo[33:65][big]) < 2e-3), k
        assert abs(fg[65] - fo[65]) < 2e-3, k
        assert np.all(np.abs(fg[66:68] - fo[66:68]) < 1e-5), k
        assert np.all(fg[68:] == 0.0)
        s1 = 10.0 ** fo[66]
        e_gpu = errs[k - 1](s1 * 10.0 ** Lg[k - 1])
        e_ref = errs[k - 1](lam_o[k - 1])
        assert e_gpu <= e_ref * (1 + 1e-3), (k, e_gpu, e_ref)


def test_learned_rule_evaluates_the_network_and_falls_back_to_gcv():
    """rule="learned": lambda_k = sigma_1 10^net(features_k), the same value the batch
    forward kernel gives for the features the solve reports; a network with a NaN output
    makes every step fall back to GCV, with GCV's lambda."""
    import torch
    from paper_2602_17892_gb300 import ab_gmres_hybrid
    from paper_2602_17892_gb300._binding import ct_mlp_forward
    geom = synth.parallel2d(48, 40, 71)
    K = 10
    x_true, b, _ = problem(geom, 41, 0.02, 42)
    G = gpu_geom(geom)
    rng = np.random.Generator(np.random.PCG64(43))
    v = (0.05 * rng.standard_normal(NP)).astype(np.float32)
    v[B3] = -2.0                                   # b3: outputs near log10(lambda/sigma_1) = -2
    P = to_dev(v)
    feats = torch.zeros((K, 80), dtype=torch.float32, device="cuda")
    x = torch.empty(G.n, dtype=torch.float32, device="cuda")
    out = ab_gmres_hybrid(G, to_dev(b), x, max_iters=K, rule="learned", lambda_net=P,
                          features=feats)
    assert out["lambda_fallback_steps"] == 0
    pred = torch.empty(K, dtype=torch.float32, device="cuda")
    ct_mlp_forward(P, feats, pred, bf16=True)
    torch.cuda.synchronize()
    pred = np.clip(pred.cpu().numpy().astype(np.float64), -8.0, 0.0)
    log_s1 = feats[:, 66].cpu().numpy().astype(np.float64)
    got = np.log10(out["lambdas"]) - log_s1
    assert np.all(np.abs(got - pred) < 1e-5), (got, pred)
    # NaN network -> GCV at every step
    Pn = P.clone()
    Pn[B3] = float("nan")
    outn = ab_gmres_hybrid(G, to_dev(b), x, max_iters=K, rule="learned", lambda_net=Pn)
    xg = torch.empty_like(x)
    outg = ab_gmres_hybrid(G, to_dev(b), xg, max_iters=K, rule="gcv")
    assert outn["lambda_fallback_steps"] == K
    np.testing.assert_allclose(outn["lambdas"], outg["lambdas"], rtol=1e-12)
    assert rel(x.cpu().numpy(), xg.cpu().numpy()) <= 1e-6


def test_trained_network_beats_gcv_on_held_out_problems():
    """The committed network, trained by the library's own kernels on solves that the library
    generated, against GCV on problems outside its training seeds: smaller mean reconstruction
    error, never a GCV fallback, and per problem no worse than GCV's error + 2 % (relative) on
    at least three quarters of the held-out problems."""
    from paper_2602_17892_gb300.lambda_net import compare_rules, load_params
    P, meta = load_params()
    seeds = np.arange(20_000_000, 20_000_000 + 12)
    r = compare_rules(P, seeds)
    learned, gcv = np.asarray(r["learned"]), np.asarray(r["gcv"])
    assert r["fallback_steps"] == 0
    assert learned.mean() < gcv.mean(), (learned, gcv, r)
    ok = int(np.sum(learned <= 1.02 * gcv))
    assert ok >= int(np.ceil(0.75 * len(seeds))), (ok, learned / gcv)
