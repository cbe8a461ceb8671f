"""Learned warm start: training data from the plain solver's own trajectories, training
with the library's kernels, and evaluation against the plain solve.

The paper starts each frame from the previous frame's warp (Sec. 7.1).  Here a U-Net
(vd_unet_*) maps (u_{f-1} / h, scaled data-term gradient of frame f at u_{f-1}) to the
increment (u_f - u_{f-1}) / h that the plain flip-flop solve of frame f produced, on
synthetic sequences of three bent capsules whose joint angles random-walk by up to 5
degrees per frame (synth.sequence_frames).  At run time vd_warm_start adds the
prediction (kept only if it lowers E_total), and the plain solve then runs until it
reaches the plain solve's own final energy (vd_set_energy_target), at most the same
schedule; if it does not get there, the plain solve from the previous warp is the
fallback.

Everything here is plumbing around the C ABI: the features, the network's forward and
backward passes, Adam and the solves run in the library's CUDA kernels; torch only holds
device buffers and events.

  python -m paper_1603_08161_b300.learned train --seeds 1-192 --frames 17 --epochs 16 --out w.bin
  python -m paper_1603_08161_b300.learned eval --weights w.bin --seeds 10001-10004
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import synth

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_capsules96.bin")
GN_ITERS, CG_ITERS = 10, 20       # the config-2 schedule
E_RTOL = 1e-5                     # "same final energy": E <= E_plain (1 + 1e-5)


def _seeds(spec):
    out = []
    for part in str(spec).split(","):
        if "-" in part:
            a, b = part.split("-")
            out += list(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    return out


def solve_params(vd, **kw):
    return vd.params(gn_iters=GN_ITERS, cg_iters=CG_ITERS, **kw)


class Tracker:
    """One all-nodes lattice on its own torch stream, with device copies of the warp."""

    def __init__(self, vd, torch, fr):
        self.vd, self.torch = vd, torch
        self.stream = torch.cuda.Stream()
        self.lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL, stream=self.stream.cuda_stream)
        self.nn = self.lat.nn
        self.h = float(fr.spacing)
        self.dims = fr.dims

    def state(self):
        t = self.torch
        u = t.empty((self.nn, 3), device="cuda")
        R = t.empty((self.nn, 9), device="cuda")
        self.lat.get_warp(u, R)
        return u, R

    def restore(self, st):
        self.lat.set_warp(st[0], st[1])

    def frame(self, fr):
        self.lat.set_frame_from(fr, "cuda")


def _frames(seeds, frames, workers, render):
    """Sequences traced on the GPU ("cuda") or by numpy in a process pool (None)."""
    return synth.sequences(seeds, frames, workers, device=render)


def collect(seeds, frames, workers=1, max_samples=None, log=print, render="cuda"):
    """(inputs, targets): lists of CUDA tensors (nn x 6, nn x 3), one pair per frame
    f >= 1 of each sequence, along the plain solver's trajectory."""
    import torch
    from . import vd
    X, T = [], []
    tr = None
    t0 = time.time()
    for seed, frs in _frames(seeds, frames, workers, render):
        if tr is None:
            tr = Tracker(vd, torch, frs[0])
        tr.frame(frs[0])
        tr.lat.solve(solve_params(vd, init=vd.VD_INIT_ZERO))
        u_prev = torch.empty((tr.nn, 3), device="cuda")
        u = torch.empty((tr.nn, 3), device="cuda")
        for fr in frs[1:]:
            tr.frame(fr)
            x = torch.empty((tr.nn, 6), device="cuda")
            tr.lat.warm_features(solve_params(vd), out=x)
            tr.lat.get_warp(u_prev)
            tr.lat.solve(solve_params(vd))
            tr.lat.get_warp(u)
            X.append(x)
            T.append((u - u_prev) / tr.h)
            if max_samples and len(X) >= max_samples:
                return X, T, tr.dims
        log(f"sequence {seed}: {len(X)} samples, {time.time() - t0:.0f} s")
    return X, T, tr.dims


def train(X, T, dims, epochs=6, lr=1e-3, surface_weight=9.0, seed=0, val=0.1, log=print):
    """Adam with a cosine learning-rate decay, one 96^3 volume per step; nodes that carry
    data (non-zero gradient input) weigh 1 + surface_weight in the loss."""
    from . import vd
    net = vd.UNet(dims, seed=seed)
    n = len(X)
    nv = max(1, int(round(val * n))) if n > 1 else 0
    tr_idx, va_idx = np.arange(n - nv), np.arange(n - nv, n)
    rng = np.random.default_rng(seed)
    steps, k = epochs * len(tr_idx), 0
    hist = []
    for ep in range(epochs):
        tl = []
        for i in rng.permutation(tr_idx):
            a = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(steps, 1)))
            tl.append(net.train_step(X[i], T[i], a, surface_weight))
            k += 1
        vl = [net.train_step(X[i], T[i], 0.0, surface_weight) for i in va_idx]
        base = []
        for i in va_idx:  # the loss of a zero prediction, same weights
            w = 1.0 + surface_weight * (X[i][:, 3:].abs().sum(1, keepdim=True) > 0).float()
            base.append(float((w * T[i] ** 2).mean()))
        hist.append({"epoch": ep, "train_loss": float(np.mean(tl)), "val_loss": float(np.mean(vl)) if vl else None,
                     "val_zero_loss": float(np.mean(base)) if base else None})
        log(json.dumps(hist[-1]))
    return net, hist


def evaluate(net, seeds, frames, workers=1, log=print, render="cuda"):
    """Per frame f >= 1 of each sequence, from the plain trajectory's warp of frame f-1:
    the plain solve (full schedule) sets E_plain; then the plain solve and the learned
    start are each run until E <= E_plain (1 + 1e-5).  Times are CUDA events on the
    lattice's stream (set_warp and frame upload excluded)."""
    import torch
    from . import vd
    tr = None
    rec = []
    for seed, frs in _frames(seeds, frames, workers, render):
        if tr is None:
            tr = Tracker(vd, torch, frs[0])
        lat = tr.lat
        # one gated graph for every solve: only the target's value changes below (a
        # target of 0 is never met, so that solve runs the full schedule)
        lat.set_energy_target(0.0)
        tr.frame(frs[0])
        lat.solve(solve_params(vd, init=vd.VD_INIT_ZERO))
        lat.warm_features(solve_params(vd), out=torch.empty((tr.nn, 6), device="cuda"))  # allocates
        for fi, fr in enumerate(frs[1:], 1):
            tr.frame(fr)
            prev = tr.state()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

            def timed(fn):
                torch.cuda.synchronize()
                ev[0].record(tr.stream)
                out = fn()
                ev[1].record(tr.stream)
                ev[1].synchronize()
                return out, ev[0].elapsed_time(ev[1])

            def plain():
                lat.solve_async(solve_params(vd))
                return lat.report()

            def learned():
                lat.warm_start(net, solve_params(vd), wait=False)
                lat.solve_async(solve_params(vd))
                return lat.report()

            lat.set_energy_target(0.0)
            rp, t_plain = timed(plain)
            plain_state = tr.state()
            target = rp["e_total"] * (1.0 + E_RTOL)
            lat.set_energy_target(target)
            tr.restore(prev)
            rs, t_stop = timed(plain)
            tr.restore(prev)
            rl, t_learn = timed(learned)
            wr = lat.warm_report()
            fallback = not (rl["e_total"] <= target)
            if fallback:  # the plain solve from the previous warp
                tr.restore(prev)
                lat.set_energy_target(0.0)
                _, t_fb = timed(plain)
                t_learn += t_fb
            rec.append({"seed": seed, "frame": fi, "e_plain": rp["e_total"], "e_learned": rl["e_total"],
                        "gn_plain_stop": rs["gn_done"], "gn_learned": rl["gn_done"], "ms_plain": t_plain,
                        "ms_plain_stop": t_stop, "ms_learned": t_learn, "used_prediction": wr["used_prediction"],
                        "e_start": wr["e_start"], "e_predicted": wr["e_predicted"], "fallback": fallback})
            tr.restore(plain_state)
            log(json.dumps(rec[-1]))
    return summarize(rec), rec


def summarize(rec):
    n = len(rec)
    s = lambda k: float(sum(r[k] for r in rec))
    return {"frames": n,
            "fps_plain": 1e3 * n / s("ms_plain"),
            "fps_plain_same_tolerance": 1e3 * n / s("ms_plain_stop"),
            "fps_learned": 1e3 * n / s("ms_learned"),
            "gn_mean_plain_same_tolerance": s("gn_plain_stop") / n,
            "gn_mean_learned": s("gn_learned") / n,
            "prediction_used": s("used_prediction") / n,
            "fallbacks": int(s("fallback")),
            "e_predicted_over_e_start": float(np.median([r["e_predicted"] / r["e_start"] for r in rec]))}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("cmd", choices=["train", "eval", "time"])
    ap.add_argument("--iters", type=int, default=10, help="time: forward passes and training steps timed")
    ap.add_argument("--seeds", default=None)
    ap.add_argument("--frames", type=int, default=17)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--surface-weight", type=float, default=9.0)
    ap.add_argument("--max-samples", type=int, default=None)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--log", default=None)
    ap.add_argument("--cpu-render", action="store_true", help="trace the frames with numpy in a process pool")
    a = ap.parse_args(argv)
    logf = open(a.log, "a") if a.log else None

    def log(msg):
        print(msg, flush=True)
        if logf:
            logf.write(msg + "\n")
            logf.flush()

    if a.cmd == "time":  # the network alone at 96^3 (random input), CUDA-event timed
        import torch
        from . import vd
        dims = synth.lattice_for(96)[0]
        net = vd.UNet(dims, seed=1)
        n = int(np.prod(dims))
        x = torch.randn((n, 6), device="cuda")
        t = 0.1 * torch.randn((n, 3), device="cuda")
        o = torch.empty((n, 3), device="cuda")
        out = {}
        for name, fn in (("forward_ms", lambda: net.forward(x, o)), ("train_step_ms", lambda: net.train_step(x, t, 1e-4))):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(a.iters):
                fn()
            torch.cuda.synchronize()
            out[name] = (time.perf_counter() - t0) * 1e3 / a.iters
        log(json.dumps(out))
    elif a.cmd == "train":
        seeds = _seeds(a.seeds or "1-192")
        X, T, dims = collect(seeds, a.frames, a.workers, a.max_samples, log, None if a.cpu_render else "cuda")
        log(json.dumps({"samples": len(X)}))
        net, _ = train(X, T, dims, a.epochs, a.lr, a.surface_weight, log=log)
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        net.save(a.out)
        log(json.dumps({"saved": a.out}))
    else:
        from . import vd
        seeds = _seeds(a.seeds or "10001-10004")
        dims = synth.lattice_for(96)[0]
        net = vd.UNet(dims)
        net.load(a.weights)
        summ, _ = evaluate(net, seeds, a.frames, a.workers, log, None if a.cpu_render else "cuda")
        log(json.dumps(summ))


if __name__ == "__main__":
    main()
