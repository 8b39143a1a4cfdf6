"""Inverse design of the grating-coupler analogue (the paper's Sec. 4 / Fig. 4).

Parameters theta in [0, 1] on the dev x dev grid of the design region:

    theta -> Gaussian filter (60 nm = 3 cells at 20 nm) -> projection of
    sharpness beta (beta = 1 for the first 40 iterations, then beta_max)
    -> rho -> eps = SiO2 + (Si - SiO2) rho, extruded over the 220 nm layer
    -> FDTD time loop with the compressed boundary tape -> (L, M)
    -> transmission T = -L / M (flux along +x through the output waveguide
       over the downward flux above the device)

and the loss -10 log10(T) is minimised with Adam with Nesterov momentum
(torch.optim.NAdam) and a linear learning-rate warm-up; theta is clipped to
[0, 1] after every step.  The gradient of (L, M) comes from one time-reversed
run per iteration (`fdtd.objectives`); the filter and the projection are
plain torch operations in front of it.

The paper's projection is a subpixel-smoothed projection that stays
differentiable at beta = infinity; here a tanh projection with a large
finite beta_max stands in for it.

    python -m paper_2603_24027_gb300.design --tape e4m3b11fnuz:16:linear --seeds 0 1 2 \
        --iters 200 --out runs.jsonl
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch
import torch.nn.functional as Fn

from . import _capi as A
from . import fdtd
from . import inputs as I


def gaussian_filter2d(x: torch.Tensor, sigma: float) -> torch.Tensor:
    """Separable Gaussian blur of a 2D field with edge replication."""
    r = int(math.ceil(3.0 * sigma))
    t = torch.arange(-r, r + 1, dtype=x.dtype, device=x.device)
    k = torch.exp(-0.5 * (t / sigma) ** 2)
    k = k / k.sum()
    y = Fn.pad(x[None, None], (r, r, r, r), mode="replicate")
    y = Fn.conv2d(y, k.view(1, 1, 1, -1))
    y = Fn.conv2d(y, k.view(1, 1, -1, 1))
    return y[0, 0]


def project(rho: torch.Tensor, beta: float, eta: float = 0.5) -> torch.Tensor:
    """Smoothed Heaviside of sharpness beta around threshold eta (tanh form)."""
    a = math.tanh(beta * eta)
    return (a + torch.tanh(beta * (rho - eta))) / (a + math.tanh(beta * (1.0 - eta)))


class Coupler:
    """One coupler problem: workload, simulation handle and tape settings."""

    def __init__(self, workload=None, rec=None, device="cuda", sigma_cells: float = 3.0):
        self.w = workload if workload is not None else I.coupler()
        self.rec = rec if rec is not None else A.record_cfg("f32", 1)
        self.sim = fdtd.Simulation(self.w, device=torch.device(device))
        self.eps_bg = torch.from_numpy(self.w.eps).to(device)
        lo, hi = self.w.design_lo, self.w.design_hi
        self.shape2d = (hi[1] - lo[1], hi[0] - lo[0])
        self.layer = hi[2] - lo[2]
        self.sigma = sigma_cells

    def rho(self, theta: torch.Tensor, beta: float) -> torch.Tensor:
        return project(gaussian_filter2d(theta, self.sigma), beta)

    def eps_design(self, theta: torch.Tensor, beta: float) -> torch.Tensor:
        r = self.rho(theta, beta)
        e = I.EPS_SIO2 + (I.EPS_SI - I.EPS_SIO2) * r
        return e[None].expand(self.layer, *self.shape2d)

    def transmission(self, theta: torch.Tensor, beta: float) -> torch.Tensor:
        """T = -L / M as a differentiable float64 scalar."""
        LM = fdtd.objectives(self.eps_design(theta, beta), self.eps_bg, self.sim, self.rec)
        return -LM[0] / LM[1]


def optimise(problem: Coupler, theta0: np.ndarray, iters: int = 200, lr: float = 0.02,
             warmup: int = 20, beta_switch: int = 40, beta_max: float = 64.0, log=None):
    """NAdam on -10 log10(T); returns (theta, history of T in dB)."""
    dev = problem.eps_bg.device
    theta = torch.tensor(theta0, dtype=torch.float64, device=dev, requires_grad=True)
    opt = torch.optim.NAdam([theta], lr=lr)
    sched = torch.optim.lr_scheduler.LambdaLR(opt, lambda i: min(1.0, (i + 1) / warmup))
    hist = []
    for it in range(iters):
        beta = 1.0 if it < beta_switch else beta_max
        opt.zero_grad()
        T = problem.transmission(theta, beta)
        tdb = 10.0 * torch.log10(torch.clamp(T, min=1e-12))
        (-tdb).backward()
        opt.step()
        sched.step()
        with torch.no_grad():
            theta.clamp_(0.0, 1.0)
        hist.append(float(tdb.detach()))
        if log:
            log(it, float(tdb.detach()), beta)
    # transmission of the final, fully projected design
    with torch.no_grad():
        final = float(10.0 * torch.log10(torch.clamp(problem.transmission(theta, beta_max),
                                                       min=1e-12)))
    return theta.detach(), hist, final


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--tape", default="f32:1:linear")
    p.add_argument("--seeds", type=int, nargs="+", default=[0])
    p.add_argument("--iters", type=int, default=200)
    p.add_argument("--lr", type=float, default=0.02)
    p.add_argument("--steps", type=int, default=2000, help="time steps per simulation")
    p.add_argument("--out", default=None)
    a = p.parse_args(argv)
    from . import build as B
    B.build()
    dt, k, interp = a.tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    rows = []
    for seed in a.seeds:
        w = I.coupler(n_steps=a.steps)
        prob = Coupler(w, rec)
        theta0 = np.random.default_rng(seed).uniform(0.0, 1.0, prob.shape2d)
        t0 = time.perf_counter()
        _, hist, final = optimise(prob, theta0, iters=a.iters, lr=a.lr)
        row = dict(tape=a.tape, seed=seed, iters=a.iters, initial_db=hist[0], best_db=max(hist),
                   final_db=final, seconds=time.perf_counter() - t0, history_db=hist)
        rows.append(row)
        print(json.dumps({k_: v for k_, v in row.items() if k_ != "history_db"}), flush=True)
    if a.out:
        with open(a.out, "a") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")


if __name__ == "__main__":
    main()
