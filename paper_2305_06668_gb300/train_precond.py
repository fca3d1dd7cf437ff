"""Train the learned preconditioner scale on the GPU with the library's own kernels.

Data: FP64 LOBPCG runs (diagonal preconditioner) on seeded matrices of two families,
  * "cfg1": sparse_cfg1 recipe (diagonal 0.01 i + U(0, 0.005), 16 random couplings per
    row, N(0, 0.01^2)), k = 4,
  * "ci":   sparse_ci recipe (diagonal 0.001 i + U(0, 0.01), banded + long-range
    couplings N(0, 0.005^2)), k = 16 with 5 extra block vectors,
both at n = 200,000.  For each matrix the converged eigenvectors x* are computed first;
then runs stopped after t iterations (same initial block) give Ritz pairs (theta, x).
For every sought column the exact correction e = x* - x (x* sign-aligned, projected
orthogonal to x) is the target direction; the loss is 1 - cos^2(w, e) per column with
w = s r / (d - theta) (s = 1 outside the learned region).

Every arithmetic step (products with A, Gram, features, forward, loss, backward, Adam)
runs in the library's CUDA kernels; PyTorch only holds device memory.

Usage: python -m paper_2305_06668_gb300.train_precond --out weights.npy [--train 100 --heldout 10]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import sys
import time

import numpy as np

FAMILIES = {"cfg1": dict(k=4, extra=0, snapshots=(1, 2, 3, 5)),
            "ci": dict(k=16, extra=5, snapshots=(3, 10, 30, 100))}


@dataclasses.dataclass
class Columns:
    F: object
    q: object
    e: object
    col: object
    ee: object
    far_we: object
    far_ww: object


def make_matrix(family: str, n: int, seed: int):
    import synth
    return synth.sparse_cfg1(n=n, seed=seed) if family == "cfg1" else synth.sparse_ci(n=n, seed=seed)


def harvest(lb, torch, family: str, n: int, seed: int, xstar_maxiter: int = 4000, bootstrap=None):
    """Training columns of one matrix (near rows only) or None if the reference solve fails.

    bootstrap: parameters of an earlier model, used only to reach the converged x*
    faster (the snapshots always come from diagonal-preconditioned runs)."""
    import synth
    spec = FAMILIES[family]
    k, extra = spec["k"], spec["extra"]
    a = make_matrix(family, n, seed)
    t = lb.upload_csr(a)
    x0 = torch.from_numpy(synth.diag_guess(a.diag, k + extra, seed=seed, noise=0.0)).cuda()
    kw = dict(precond=lb.PREC_LEARNED, mlp_weights=bootstrap) if bootstrap is not None else {}
    ref = lb.Solver(**t, extra=extra, maxiter=xstar_maxiter, **kw).solve(k, 1e-7, X0=x0)
    if ref.status != lb.OK:
        return None
    XS = ref.evecs.contiguous()  # n x k row-major
    rho, cscale = lb.row_norms(a.n, row_ptr=t["row_ptr"], col_idx=t["col_idx"], val=t["val"])
    out = []
    for it in spec["snapshots"]:
        r = lb.Solver(**t, extra=extra, maxiter=it).solve(k, 1e-7, X0=x0)
        if r.status == lb.OK:
            continue  # already converged: nothing left to correct
        X = r.evecs.contiguous()
        AX = lb.spmm_csr(t["row_ptr"], t["col_idx"], t["val"], X)
        lam = torch.from_numpy(r.evals).cuda()
        G = lb.gram(X, XS)  # k x k, alpha_j = x_j . x*_j on the diagonal
        alpha = torch.diagonal(G).contiguous()
        sign = torch.where(alpha < 0, -1.0, 1.0).to(torch.float64)
        XSa = (XS * sign[None, :]).contiguous()
        alpha = alpha * sign
        colmax = (AX - X * lam[None, :]).abs().amax(dim=0).contiguous()
        F, q, e, near, ee, far_we, far_ww = lb.precond_features(X, AX, lam, t["diag"], rho, cscale, colmax, XSa, alpha)
        # drop columns that are already converged (no direction to learn)
        keep_col = (ee > 1e-24)
        idx = torch.nonzero(near.bool()).squeeze(1)
        colid = (idx % k).to(torch.int32)
        sel = keep_col[colid.long()]
        idx, colid = idx[sel], colid[sel]
        out.append((F[idx], q[idx], e[idx], colid, ee, far_we, far_ww, keep_col))
    return out, float(cscale)


def assemble(torch, pieces):
    """Concatenate harvested snapshots into one column-indexed training set."""
    Fs, qs, es, cols, ees, fws, fwws = [], [], [], [], [], [], []
    base = 0
    for F, q, e, colid, ee, far_we, far_ww, keep in pieces:
        kept = torch.nonzero(keep).squeeze(1)
        remap = torch.full((ee.numel(),), -1, dtype=torch.int64, device=ee.device)
        remap[kept] = torch.arange(kept.numel(), device=ee.device)
        Fs.append(F), qs.append(q), es.append(e)
        cols.append((remap[colid.long()] + base).to(torch.int32))
        ees.append(ee[kept]), fws.append(far_we[kept]), fwws.append(far_ww[kept])
        base += kept.numel()
    cat = lambda v: torch.cat(v).contiguous()
    return Columns(cat(Fs), cat(qs), cat(es), cat(cols), cat(ees), cat(fws), cat(fwws))


def init_params(num: int, seed: int = 0) -> np.ndarray:
    """He-style initialisation; b3 = log(e - 1) so that softplus(z) starts near 1."""
    g = np.random.default_rng(seed)
    P = np.zeros(num, dtype=np.float32)
    H = 64
    P[0:3 * H] = g.normal(0, np.sqrt(2 / 3), 3 * H)
    P[4 * H:4 * H + H * H] = g.normal(0, np.sqrt(2 / H), H * H)
    P[5 * H + H * H:6 * H + H * H] = g.normal(0, 0.01, H)
    P[-1] = np.log(np.e - 1)
    return P


def loss_of(lb, torch, P, data: Columns) -> float:
    s = lb.mlp_forward(data.F, P)
    loss, _ = lb.mlp_loss(data.col, data.q, data.e, s, data.far_we, data.far_ww, data.ee)
    return loss


def baseline_loss(lb, torch, data: Columns) -> float:
    """Loss of the plain diagonal preconditioner (s = 1 everywhere)."""
    s = torch.ones_like(data.q)
    loss, _ = lb.mlp_loss(data.col, data.q, data.e, s, data.far_we, data.far_ww, data.ee)
    return loss


def train(lb, torch, data: Columns, epochs: int, lr: float, seed: int = 0, log=print):
    P = torch.from_numpy(init_params(lb.mlp_num_params(), seed)).cuda()
    grad, m, v = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
    hist = []
    for ep in range(1, epochs + 1):
        s = lb.mlp_forward(data.F, P)
        loss, d = lb.mlp_loss(data.col, data.q, data.e, s, data.far_we, data.far_ww, data.ee)
        lb.mlp_backward(data.F, P, d, grad)
        lb.mlp_adam(P, grad, m, v, ep, lr=lr)
        hist.append(loss)
        if ep == 1 or ep % 50 == 0 or ep == epochs:
            log(f"epoch {ep}: loss {loss:.5f}")
    return P.cpu().numpy(), hist


def evaluate(lb, torch, weights: np.ndarray, n: int, seeds: dict, maxiter: int = 4000, precision=None):
    """Solve held-out matrices with the diagonal and with the learned preconditioner.

    Returns one record per matrix: iterations, time, final max residual and the largest
    eigenvalue difference between the two runs."""
    import synth
    precision = lb.FP64 if precision is None else precision
    rows = []
    for fam, fam_seeds in seeds.items():
        spec = FAMILIES[fam]
        k, extra = spec["k"], spec["extra"]
        for seed in fam_seeds:
            a = make_matrix(fam, n, seed)
            t = lb.upload_csr(a)
            x0 = torch.from_numpy(synth.diag_guess(a.diag, k + extra, seed=seed, noise=0.0)).cuda()
            rec = {"family": fam, "seed": seed}
            ev = {}
            for name, pc in (("diag", lb.PREC_DIAG), ("learned", lb.PREC_LEARNED)):
                kw = dict(mlp_weights=weights) if pc == lb.PREC_LEARNED else {}
                s = lb.Solver(**t, extra=extra, maxiter=maxiter, precond=pc, precision=precision, **kw)
                r = s.solve(k, 1e-8, X0=x0)
                s.close()
                rec[name] = {"status": lb.STATUS_NAMES[r.status], "iterations": r.info["iterations"],
                             "seconds": r.info["seconds"], "max_res": float(np.max(r.resnorms)),
                             "fallback": r.info["precond_fallback"]}
                ev[name] = r.evals
            rec["max_rel_eig_diff"] = float(np.max(np.abs(ev["learned"] - ev["diag"]) / np.maximum(1, np.abs(ev["diag"]))))
            rows.append(rec)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--train", type=int, default=100, help="matrices per family for training")
    ap.add_argument("--heldout", type=int, default=10, help="matrices per family held out")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--report", default=None, help="JSON summary path")
    ap.add_argument("--bootstrap", default=None, help="earlier weights (.npy) used to compute x* faster")
    args = ap.parse_args(argv)
    import torch

    import paper_2305_06668_gb300 as lb
    t0 = time.time()
    boot = np.load(args.bootstrap).astype(np.float32) if args.bootstrap else None
    train_pieces, held_pieces = [], []
    for fam in FAMILIES:
        for i in range(args.train + args.heldout):
            seed = 1000 * (1 + list(FAMILIES).index(fam)) + i
            res = harvest(lb, torch, fam, args.n, seed, bootstrap=boot)
            if res is None:
                print(f"{fam} seed {seed}: reference solve did not converge, skipped", file=sys.stderr)
                continue
            (held_pieces if i >= args.train else train_pieces).extend(res[0])
        print(f"harvested {fam}: {time.time() - t0:.0f} s", file=sys.stderr, flush=True)
    tr = assemble(torch, train_pieces)
    ho = assemble(torch, held_pieces)
    print(f"training samples {tr.q.numel()}, columns {tr.ee.numel()}; held-out columns {ho.ee.numel()}",
          file=sys.stderr)
    P, hist = train(lb, torch, tr, args.epochs, args.lr, log=lambda m: print(m, file=sys.stderr, flush=True))
    Pd = torch.from_numpy(P).cuda()
    summary = {"train_samples": int(tr.q.numel()), "train_columns": int(tr.ee.numel()),
               "heldout_columns": int(ho.ee.numel()), "loss_train_diag": baseline_loss(lb, torch, tr),
               "loss_train_learned": loss_of(lb, torch, Pd, tr), "loss_heldout_diag": baseline_loss(lb, torch, ho),
               "loss_heldout_learned": loss_of(lb, torch, Pd, ho), "epochs": args.epochs, "lr": args.lr,
               "n": args.n, "train_per_family": args.train, "heldout_per_family": args.heldout,
               "seconds": time.time() - t0}
    np.save(args.out, P.astype(np.float32))
    held = {fam: [1000 * (1 + list(FAMILIES).index(fam)) + i for i in range(args.train, args.train + args.heldout)]
            for fam in FAMILIES}
    summary["heldout_solves"] = evaluate(lb, torch, P.astype(np.float32), args.n, held)
    for fam in FAMILIES:
        recs = [r for r in summary["heldout_solves"] if r["family"] == fam]
        if recs:
            summary[f"heldout_{fam}_mean_iterations"] = {
                name: float(np.mean([r[name]["iterations"] for r in recs])) for name in ("diag", "learned")}
    print(json.dumps(summary), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(summary, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
