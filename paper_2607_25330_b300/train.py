"""Physics-informed training of the factorised FNO on synthetic Manhattan masks.

The loss is the paper's physics residual of Sec. 3 (Eq. loss: the squared PSFD residual
|A G_theta(a) - b|^2 plus the weighted high-frequency term), with the PSFD operator and its
adjoint from the library and the FNO forward and reverse passes from the library; the parameters
are updated with Adam.  `train` loops the step over a pool of seeded masks and `evaluate` measures
what the warm start is for: the initial relative residual of the FNO prediction and the
iterations a solve needs from it, against the seed-initialised network, on held-out masks.

    python -m paper_2607_25330_b300.train --steps 600 --batch 8

Run on the GPU; prints one JSON line.
"""
import argparse
import json
import time
from typing import Dict, List

import numpy as np
import torch

from . import inputs as I
from . import psfd
from .autograd import fno_apply, physics_loss


def _weights(seed: int, zero_output: bool = False) -> Dict[str, torch.Tensor]:
    """Seed-initialised parameters; zero_output starts the last projection layer at zero, so that
    the untrained network predicts E = 0 (the cold start) and training only improves on it."""
    S = I.FNOShape()
    w = I.fno_weights(S, seed, spectral_scale=1.0)
    if zero_output:
        w["q2"] = np.zeros_like(w["q2"])
        w["qb2"] = np.zeros_like(w["qb2"])
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda().requires_grad_(True) for k, v in w.items()}


def train(steps: int, batch: int, lr: float, pool: int, seed: int, preset: str, log_every: int = 10,
          pol: int = None, mask_seed: int = 1000, zero_output: bool = False, w: Dict = None,
          mask_kind: str = None):
    """Adam on the physics loss over `pool` seeded masks (a random batch of them per step); `pol`
    selects the illumination (one model per polarisation), default the preset's first; `w`
    continues from given parameters."""
    prob = I.preset(preset)
    prob.pols = [prob.pols[0] if pol is None else int(pol)]
    S = I.FNOShape()
    if w is None:
        w = _weights(seed, zero_output)
    trainer = psfd.FnoTrainer(psfd.fno_struct(w, S), batch, prob.nz, prob.ny, prob.nx, checkpoint=True)
    plans = [psfd.Plan(prob, nrhs=1) for _ in range(batch)]
    masks = [torch.from_numpy(I.mask_for(prob, mask_seed + i, mask_kind)) for i in range(pool)]
    stack, zprof = prob.stack(), prob.zprofile()
    opt = torch.optim.Adam(list(w.values()), lr=lr)
    rng = np.random.default_rng(seed)
    log: List[Dict] = []
    t0 = time.time()
    for step in range(steps):
        idx = rng.choice(pool, size=batch, replace=False)
        fills, bs = [], []
        for s, i in enumerate(idx):
            fill = plans[s].mask_fill(masks[i], zprof)
            bs.append(plans[s].background(stack, fill, prob.pols))
            fills.append(fill)
        a = torch.stack(fills).contiguous()
        opt.zero_grad(set_to_none=True)
        E = fno_apply(trainer, w, a)
        J = sum(physics_loss(plans[s], E[s:s + 1], bs[s]) for s in range(batch)) / batch
        J.backward()
        opt.step()
        if step % log_every == 0 or step == steps - 1:
            log.append({"step": step, "loss": float(J.detach()), "s": time.time() - t0})
    return w, log


def evaluate(w: Dict[str, torch.Tensor], preset: str, masks: int, tol: float = 1e-6, pol: int = None) -> Dict:
    """Warm start from the network on held-out masks: initial relative residual and BiCGSTAB
    iterations to `tol` with the layered preconditioner (mean over masks)."""
    prob = I.preset(preset)
    prob.pols = [prob.pols[0] if pol is None else int(pol)]
    S = I.FNOShape()
    ws = psfd.fno_struct({k: v.detach() for k, v in w.items()}, S)
    plan = psfd.Plan(prob, nrhs=1)
    r0, its = [], []
    built = False
    for m in range(masks):
        fill = plan.mask_fill(torch.from_numpy(I.mask_for(prob, 9000 + m)), prob.zprofile())
        b = plan.background(prob.stack(), fill, prob.pols)
        if not built:
            plan.layered_storage(True)
            plan.layered_build()
            built = True
        else:
            plan.layered_refresh(0.25)
        x0 = psfd.fno_forward(ws, fill.unsqueeze(0).contiguous())
        res = plan.solve_ex(b, x0=x0, tol=tol, maxit=600, method=psfd.PSFD_BICGSTAB, precond=psfd.PC_LAYERED,
                            refine=True, inner_tol=1e-3)
        info = res["info"][0]
        r0.append(info["r_rel_initial"])
        its.append(info["iters"])
    return {"r_rel_initial": float(np.mean(r0)), "iters": float(np.mean(its)), "masks": masks}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--pool", type=int, default=128)
    ap.add_argument("--seed", type=int, default=91)
    ap.add_argument("--preset", default="fno_train_128x128x48")
    ap.add_argument("--eval-masks", type=int, default=8)
    args = ap.parse_args()
    before = evaluate(_weights(args.seed), args.preset, args.eval_masks)
    w, log = train(args.steps, args.batch, args.lr, args.pool, args.seed, args.preset)
    after = evaluate(w, args.preset, args.eval_masks)
    print(json.dumps({"preset": args.preset, "steps": args.steps, "batch": args.batch, "lr": args.lr,
                      "pool": args.pool, "loss": log, "held_out_seed_weights": before,
                      "held_out_trained": after}), flush=True)


if __name__ == "__main__":
    main()
