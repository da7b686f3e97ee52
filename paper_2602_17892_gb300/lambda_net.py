"""Learned lambda rule (not in the paper): training data, training and parameter files.

The network (80 features of the projected problem -> 64 -> 64 -> 1, GELU) predicts
log10(lambda_k / sigma_1(H_k)); the library computes the features inside the hybrid step and
evaluates the network there when a solve uses ``rule="learned"`` (GCV replaces a non-finite
output).  Everything numerical runs in the library's kernels:

* data: ``ct_lambda_samples`` runs one hybrid AB-GMRES solve and returns, for every step k, the
  features of H_k and the label log10(lambda*_k / sigma_1), lambda*_k the lambda that
  minimises the reconstruction error ||x_k(lambda) - x_true|| for the known phantom;
* training: ``ct_mlp_train`` (BF16 tensor-core forward and backward, FP32 Adam).

Training problems: 256 x 256 parallel-beam scans with the angular sampling of the 64 x 64
ellipse workload (90 views over [0, pi), ceil(sqrt(2) N) + 4 bins), random 10-ellipse phantoms
(seed = problem index), Gaussian noise of level eta ~ U[0.5 %, 5 %], K = 30 steps, GCV.

The network standardises its inputs in FP32 with the mean and spread of each feature over the
training set (stored with the parameters), so that BF16 rounding acts on O(1) values.

``python -m paper_2602_17892_gb300.lambda_net --solves 20000`` generates the data, trains, and
writes ``data/lambda_net_parallel256.npz`` next to this file.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import threading
import time

import numpy as np

from ._binding import (CT_MLP_NIN, CT_MLP_NPARAMS, Geom, ab_gmres_hybrid, ct_forward_A,
                       ct_lambda_samples, ct_mlp_forward, ct_mlp_train)

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PARAMS = os.path.join(_HERE, "data", "lambda_net_parallel256.npz")
N_HID = 64
K_TRAIN = 30


def training_geometry(N: int = 256, n_views: int = 90):
    import synth
    return synth.parallel2d(N, n_views)


def noise_level(seed: int) -> float:
    """eta ~ U[0.005, 0.05], drawn from the problem's seed."""
    g = np.random.Generator(np.random.PCG64([seed, 77]))
    return float(0.005 + 0.045 * g.random())


def make_problem(geom, G: Geom, seed: int, eta: float | None = None):
    """(x_true, b, noise_norm) on the device for problem `seed`: phantom and noise from the
    seeded generators, b_true = A x_true by the library's projector (on the current stream)."""
    import torch
    import synth
    eta = noise_level(seed) if eta is None else eta
    x_true = synth.ellipse_phantom(geom.nx, 10, seed=seed, ny=geom.ny, h=geom.h)
    xt = torch.from_numpy(x_true.astype(np.float32).reshape(-1)).cuda()
    bt = torch.empty(G.m, dtype=torch.float32, device="cuda")
    ct_forward_A(G, xt, bt)
    b_true = bt.cpu().numpy().astype(np.float64)
    b, e = synth.add_noise(b_true, eta, seed + 1_000_003)
    return xt, torch.from_numpy(b.astype(np.float32)).cuda(), float(np.linalg.norm(e))


def generate(seeds, geom=None, K: int = K_TRAIN, workers: int = 8, log=None):
    """Features (len(seeds) x K x 80), labels (len(seeds) x K) and the valid-step mask, all on
    the device, from one ct_lambda_samples solve per seed.  `workers` host threads each drive
    their own geometry object on their own CUDA stream."""
    import torch
    geom = training_geometry() if geom is None else geom
    n = len(seeds)
    feats = torch.zeros((n, K, CT_MLP_NIN), dtype=torch.float32, device="cuda")
    labels = torch.full((n, K), float("nan"), dtype=torch.float32, device="cuda")
    done = np.zeros(n, dtype=np.int64)
    errors = []
    nxt = [0]
    lock = threading.Lock()
    t0 = time.time()

    def work():
        try:
            G = Geom.from_geometry(geom)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                x = torch.empty(G.n, dtype=torch.float32, device="cuda")
                while True:
                    with lock:
                        i = nxt[0]
                        nxt[0] += 1
                    if i >= n:
                        break
                    xt, b, _ = make_problem(geom, G, int(seeds[i]))
                    info = ct_lambda_samples(G, b, xt, x, feats[i], labels[i], max_iters=K,
                                             rule="gcv")
                    done[i] = info["iters_done"]
                    if log and i % 1000 == 0:
                        log(f"  solve {i}/{n}  {time.time() - t0:.1f} s")
            G.close()
        except Exception as exc:      # re-raised by the caller
            errors.append(exc)

    threads = [threading.Thread(target=work) for _ in range(max(1, workers))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    torch.cuda.synchronize()
    steps = torch.arange(K, device="cuda").unsqueeze(0)
    mask = (steps < torch.from_numpy(done).cuda().unsqueeze(1)) & torch.isfinite(labels)
    return feats, labels, mask


def init_params(seed: int = 0, mu=None, sd=None) -> np.ndarray:
    """He-normal weights, zero biases, and the input standardisation (mu, 1 / sd; identity by
    default), in the library's parameter order."""
    g = np.random.Generator(np.random.PCG64(seed))
    W1 = g.standard_normal((N_HID, CT_MLP_NIN)) * math.sqrt(2.0 / CT_MLP_NIN)
    W2 = g.standard_normal((N_HID, N_HID)) * math.sqrt(2.0 / N_HID)
    w3 = g.standard_normal(N_HID) * math.sqrt(1.0 / N_HID)
    mu = np.zeros(CT_MLP_NIN) if mu is None else np.asarray(mu, np.float64)
    isd = np.ones(CT_MLP_NIN) if sd is None else 1.0 / np.asarray(sd, np.float64)
    p = np.concatenate([W1.ravel(), np.zeros(N_HID), W2.ravel(), np.zeros(N_HID), w3, [0.0],
                        mu, isd])
    assert p.size == CT_MLP_NPARAMS
    return p.astype(np.float32)


def train(X, Y, Xv=None, Yv=None, epochs: int = 40, batch: int = 4096, lr: float = 1e-3,
          seed: int = 0, log=None):
    """Adam with the library's training kernels; the standardisation (mean and spread of each
    feature over X) is part of the parameters.  Returns the FP32 parameters (numpy) and a
    history of (epoch, train loss, validation loss)."""
    import torch
    mu = X.double().mean(0)
    sd = X.double().std(0)
    sd = torch.where(sd > 1e-6, sd, torch.ones_like(sd))
    P = torch.from_numpy(init_params(seed, mu.cpu().numpy(), sd.cpu().numpy())).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    t = 0
    hist = []
    nb = (X.shape[0] + batch - 1) // batch
    for ep in range(epochs):
        step_lr = lr * (0.1 ** (ep / max(1, epochs - 1)))       # decays to lr / 10
        perm = torch.randperm(X.shape[0], device="cuda", generator=gen)
        Xp, Yp = X[perm].contiguous(), Y[perm].contiguous()
        lh = torch.empty(nb, dtype=torch.float32, device="cuda")
        t = ct_mlp_train(P, m, v, Xp, Yp, batch, 1, step_lr, t=t, loss_hist=lh)
        tr = float(lh.mean())
        va = mse(P.cpu().numpy(), Xv, Yv) if Xv is not None else float("nan")
        hist.append((ep, tr, va))
        if log:
            log(f"  epoch {ep:3d}  lr {step_lr:.2e}  train {tr:.4f}  val {va:.4f}")
    return P.cpu().numpy(), hist


def mse(params: np.ndarray, X, Y) -> float:
    """Mean squared error of the BF16 network (raw features) on the device."""
    import torch
    P = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    ct_mlp_forward(P, X.contiguous(), out)
    return float(((out - Y) ** 2).mean())


def save_params(path: str, params: np.ndarray, meta: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=np.asarray(params, dtype=np.float32), meta=json.dumps(meta))


def load_params(path: str = DEFAULT_PARAMS, device: str = "cuda"):
    """(parameters as an FP32 device tensor, metadata dict)."""
    import torch
    with np.load(path, allow_pickle=False) as z:
        p = z["params"].astype(np.float32)
        meta = json.loads(str(z["meta"]))
    if p.size != CT_MLP_NPARAMS:
        raise ValueError(f"{path}: {p.size} parameters, expected {CT_MLP_NPARAMS}")
    return torch.from_numpy(p).to(device), meta


def compare_rules(params, seeds, geom=None, K: int = K_TRAIN):
    """Relative reconstruction errors ||x_K - x_true|| / ||x_true|| of hybrid AB-GMRES with the
    learned rule, GCV and the discrepancy principle (tau = 1.01, the true noise norm) on the
    problems `seeds`, and the learned rule's GCV fallback count."""
    import torch
    geom = training_geometry() if geom is None else geom
    G = Geom.from_geometry(geom)
    out = {"learned": [], "gcv": [], "dp": [], "fallback_steps": 0}
    x = torch.empty(G.n, dtype=torch.float32, device="cuda")
    for sd in seeds:
        xt, b, nn = make_problem(geom, G, int(sd))
        nx = float(torch.linalg.vector_norm(xt))
        for rule in ("learned", "gcv", "dp"):
            info = ab_gmres_hybrid(G, b, x, max_iters=K, rule=rule, noise_norm=nn, tau=1.01,
                                   history=False, lambda_net=params if rule == "learned" else None)
            out[rule].append(float(torch.linalg.vector_norm(x - xt)) / nx)
            if rule == "learned":
                out["fallback_steps"] += info["lambda_fallback_steps"]
    G.close()
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--solves", type=int, default=20000)
    ap.add_argument("--val-solves", type=int, default=1000)
    ap.add_argument("--test-solves", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--out", default=DEFAULT_PARAMS)
    args = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)
    from .build import build
    build()
    geom = training_geometry()
    t0 = time.time()
    seeds = np.arange(args.solves + args.val_solves)
    log(f"generating {len(seeds)} solves ({geom.nx}x{geom.ny}, {geom.n_views} views, "
        f"{geom.n_det_u} bins, K={K_TRAIN})")
    F, L, M = generate(seeds, geom, workers=args.workers, log=log)
    t_gen = time.time() - t0
    ntr = args.solves
    X = F[:ntr][M[:ntr]].contiguous()
    Y = L[:ntr][M[:ntr]].contiguous()
    Xv = F[ntr:][M[ntr:]].contiguous()
    Yv = L[ntr:][M[ntr:]].contiguous()
    log(f"data: {X.shape[0]} train / {Xv.shape[0]} val samples in {t_gen:.1f} s")
    t1 = time.time()
    params, hist = train(X, Y, Xv, Yv, epochs=args.epochs, batch=args.batch, lr=args.lr, log=log)
    t_train = time.time() - t1
    test_seeds = np.arange(10_000_000, 10_000_000 + args.test_solves)
    P = torch.from_numpy(params).cuda()
    cmp = compare_rules(P, test_seeds, geom)
    summary = {k: float(np.mean(v)) for k, v in cmp.items() if k != "fallback_steps"}
    meta = dict(geometry=dict(N=geom.nx, views=geom.n_views, bins=geom.n_det_u, kind="parallel2d"),
                K=K_TRAIN, train_solves=ntr, val_solves=args.val_solves,
                train_samples=int(X.shape[0]), val_samples=int(Xv.shape[0]),
                noise="U[0.005, 0.05]", phantoms="10 ellipses, seed = problem index",
                epochs=args.epochs, batch=args.batch, lr=args.lr,
                final_train_mse=hist[-1][1], final_val_mse=hist[-1][2],
                seconds_generate=t_gen, seconds_train=t_train,
                test_seeds=[int(test_seeds[0]), int(test_seeds[-1])],
                test_mean_rel_error=summary, test_fallback_steps=cmp["fallback_steps"])
    save_params(args.out, params, meta)
    log(json.dumps(meta, indent=1))


if __name__ == "__main__":
    main()
