"""Learned scatter estimator on top of the gDRR method.

The plain method (Section 2.4 Monte Carlo + the Poisson denoiser of Section
2.5) needs many photons for a smooth scatter image.  This module trains the
library's convolutional encoder-decoder (gdrr_cnn_*) to map a cheap,
low-photon Monte Carlo scatter image plus the ray-traced primary to the
scatter image of a high-photon run, on pairs the method itself generates;
the plain method stays the reference the error is measured against.

Everything that computes runs in libgdrr kernels: Monte Carlo, ray tracing,
finalisation, denoising, scaling into the network's FP32 input, and the
network's forward, backward and Adam passes.  The error metric is the
relative l2 norm the paper uses for scatter images (Section 3.2).

Images live on the coarse scatter grid: the 512 x 384 detector of 0.776 mm
pixels binned 4 x 4, i.e. 128 x 96 pixels of 3.104 mm, simulated directly on
that grid.
"""
from __future__ import annotations

import math

import numpy as np

from . import gdrr, inputs

H, W = 96, 128
DET_PX = 0.776 * 4
SCALE = 1.0e4          # signal per source photon per pixel -> O(1) network values


def coarse_problem(seed: int, vox: float = 4.0):
    """A seeded ellipsoid torso on the coarse scatter grid."""
    return inputs.torso_problem(vox=vox, seed=seed, nu=W, nv=H, det_px=DET_PX,
                                name=f"torso-seed{seed}-{vox:g}mm-coarse")


def estimate(ctx, n: int, seed: int, angle: float, angle_index: int, length: float = 4.0, iters: int = 800):
    """The plain method at n histories on the coarse grid, one gdrr_project
    call: ray-traced primary and Poisson-denoised MC scatter (Eq. 5, omega =
    0.8) per source photon, device FP64 [H, W] each.  beta is set on the
    device so that beta times the mean count is length^2: a smoothing length
    of about `length` pixels at any photon count."""
    r = gdrr.project(ctx, n, seed, angle, bin_factor=1, smoothing_px=length, iters=iters, angle_index=angle_index)
    return r["S"], r["P"]


def network_flops(c: int = 32, h: int = H, w: int = W) -> float:
    """Convolution flops of one forward pass of one image through the
    encoder-decoder (2 x output pixels x input channels x output channels x
    kernel taps per layer): encoder 2 -> c -> 2c -> 4c -> 8c at full, 1/2, 1/4
    and 1/8 resolution, decoder (8c + 4c) -> 4c, (4c + 2c) -> 2c, (2c + c) -> c
    at 1/4, 1/2 and full resolution, then the 1 x 1 output layer c -> 1."""
    px = [h * w // (4 ** k) for k in range(4)]
    layers = [(px[0], 2, c, 9), (px[1], c, 2 * c, 9), (px[2], 2 * c, 4 * c, 9), (px[3], 4 * c, 8 * c, 9),
              (px[2], 12 * c, 4 * c, 9), (px[1], 6 * c, 2 * c, 9), (px[0], 3 * c, c, 9), (px[0], c, 1, 1)]
    return float(sum(2 * p * ci * co * k for p, ci, co, k in layers))


def plain_length(n: int) -> float:
    """Smoothing length (pixels) of the plain method's denoiser at n histories:
    12 px at 1e6 shrinking as n^-0.24 (8 px at 3e6, 7 at 1e7, 4 at 1e8), the
    lengths that minimise the error against a 2e9-history reference on
    held-out torsos (measured at 1e6, 3e6, 1e7 and 1e8)."""
    return float(min(16.0, max(2.0, 12.0 * (n / 1e6) ** -0.24)))


LOW_LENGTH = plain_length(10**6)      # the low-photon input (12 px)
HIGH_LENGTH = plain_length(10**8)     # the high-photon targets and the 1e8 comparison (4.1 px)


def low_input(ctx, n_low: int, seed: int, angle: float, angle_index: int, x_slot):
    """The network input for one projection: the plain method's low-photon
    estimate (MC + Poisson denoising) and the ray-traced primary, scaled into
    x_slot [2, H, W] FP32.  Returns the denoised low-photon estimate."""
    d_low, P = estimate(ctx, n_low, seed, angle, angle_index, plain_length(n_low))
    gdrr.gdrr_scale_to_f32(d_low, SCALE, x_slot[0])
    gdrr.gdrr_scale_to_f32(P, SCALE, x_slot[1])
    return d_low


def make_dataset(seeds, angles_per_phantom: int, n_low: int, n_high: int, rng_seed: int = 0):
    """Inputs X [N, 2, H, W] (denoised low-photon scatter, ray-traced primary)
    and targets Y [N, 1, H, W] (denoised high-photon scatter), scaled by
    SCALE, FP32; angles uniform over 360 degrees."""
    import torch
    rng = np.random.default_rng(rng_seed)
    N = len(seeds) * angles_per_phantom
    X = torch.empty((N, 2, H, W), dtype=torch.float32, device="cuda")
    Y = torch.empty((N, 1, H, W), dtype=torch.float32, device="cuda")
    k = 0
    for s in seeds:
        with gdrr.Context(coarse_problem(int(s))) as ctx:
            for a in range(angles_per_phantom):
                angle = float(rng.uniform(0.0, 2.0 * math.pi))
                low_input(ctx, n_low, 1_000_003 + 7 * k, angle, a, X[k])
                s_high, _ = estimate(ctx, n_high, 2_000_029 + 11 * k, angle, a, plain_length(n_high))
                gdrr.gdrr_scale_to_f32(s_high, SCALE, Y[k, 0])
                k += 1
    return X, Y


def train(net, X, Y, steps: int, batch: int = 16, lr: float = 1e-3, log=None):
    """Adam on consecutive batches of the (shuffled-by-construction) set,
    learning rate halved at 1/2 and 3/4 of the run.  Returns the losses."""
    N = X.shape[0]
    losses = []
    for step in range(steps):
        i0 = (step * batch) % N
        i1 = min(N, i0 + batch)
        net.forward(X[i0:i1])
        losses.append(net.backward(Y[i0:i1]))
        f = 1.0 if step < steps // 2 else (0.5 if step < 3 * steps // 4 else 0.25)
        net.adam_step(lr * f)
        if log and step % max(1, steps // 10) == 0:
            log(f"step {step} loss {losses[-1]:.5f}")
    return losses


def predict(net, X):
    """Network scatter estimate per source photon, FP64 [N, H, W] on the device."""
    import torch
    out = net.forward(X)
    S = torch.empty((X.shape[0], H, W), dtype=torch.float64, device="cuda")
    gdrr.gdrr_scale_to_f64(out, 1.0 / SCALE, S)
    return S


def rel_l2(a, ref) -> float:
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def evaluate(net, seeds=(900, 901, 902, 903), angles_per_seed=2, n_low=10**6, n_ref=2 * 10**9,
             plain_counts=(10**6, 3 * 10**6, 10**7, 10**8), rng_seed=7):
    """Held-out evaluation: relative l2 of the network's estimate and of the
    plain method at several photon counts against a denoised n_ref-history
    reference; the plain photon count that matches the network's error
    (log-log interpolation)."""
    import torch
    rng = np.random.default_rng(rng_seed)
    e_net, e_plain = [], {n: [] for n in plain_counts}
    for s in seeds:
        with gdrr.Context(coarse_problem(int(s))) as ctx:
            for a in range(angles_per_seed):
                ang = float(rng.uniform(0.0, 2.0 * math.pi))
                ref = estimate(ctx, n_ref, 91 + 10 * s + a, ang, a, 1.5)[0].cpu().numpy()
                x = torch.empty((1, 2, H, W), dtype=torch.float32, device="cuda")
                low_input(ctx, n_low, 31 + 10 * s + a, ang, a, x[0])
                e_net.append(rel_l2(predict(net, x).cpu().numpy()[0], ref))
                for n in plain_counts:
                    sp, _ = estimate(ctx, n, (31 if n < 10**8 else 57) + 10 * s + a, ang, a, plain_length(n))
                    e_plain[n].append(rel_l2(sp.cpu().numpy(), ref))
    err_net = float(np.mean(e_net))
    err_plain = {n: float(np.mean(v)) for n, v in e_plain.items()}
    lx = np.log(np.array(plain_counts, np.float64))
    ly = np.log(np.array([err_plain[n] for n in plain_counts]))
    order = np.argsort(ly)
    matched = float(np.exp(np.interp(math.log(err_net), ly[order], lx[order])))
    return {"learned": err_net, "plain": err_plain, "plain_histories_at_learned_error": matched}


def bench_network(batch: int = 64, train_batch: int = 16, reps: int = 5, channels: int = 32) -> dict:
    """Device time of the network on random inputs: a forward pass of `batch`
    images and a training step (forward, backward, Adam) of `train_batch`,
    best of `reps` after a warm-up, with the convolution flops of Section
    network_flops and the resulting TFLOP/s."""
    import torch
    net = gdrr.Cnn(max(batch, train_batch), H, W, channels, seed=1)
    x = torch.rand((batch, 2, H, W), dtype=torch.float32, device="cuda")
    t = torch.rand((train_batch, 1, H, W), dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize()
            best = min(best, ev[0].elapsed_time(ev[1]))
        return best

    def step():
        net.forward(x[:train_batch])
        net.backward(t)
        net.adam_step(1e-4)

    f_ms = timed(lambda: net.forward(x))
    s_ms = timed(step)
    net.close()
    flops = network_flops(channels)
    return {"forward_batch": batch, "forward_ms": f_ms, "forward_tflops": batch * flops / f_ms / 1e9,
            "train_batch": train_batch, "train_step_ms": s_ms,
            "train_tflops": 3 * train_batch * flops / s_ms / 1e9, "gflop_per_image": flops / 1e9}


def main(argv=None):
    """Train and evaluate the estimator at a chosen scale; prints one JSON line."""
    import argparse
    import json
    import time

    import torch
    ap = argparse.ArgumentParser(description="train the learned scatter estimator on method-generated pairs")
    ap.add_argument("--bench-network", action="store_true",
                    help="only time the network's forward pass and training step on random inputs")
    ap.add_argument("--phantoms", type=int, default=256, help="training torsos (one random angle each)")
    ap.add_argument("--steps", type=int, default=4000, help="Adam steps")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--low", type=float, default=1e6, help="histories of the network's input")
    ap.add_argument("--high", type=float, default=1e8, help="histories of the targets")
    ap.add_argument("--channels", type=int, default=32, help="base channels of the network (<= 64)")
    args = ap.parse_args(argv)
    gdrr.lib()
    if args.bench_network:
        print(json.dumps(bench_network(channels=args.channels)))
        return
    t0 = time.perf_counter()
    # training torsos from seed 10000 on; the held-out torsos are 900 ... 903
    X, Y = make_dataset(range(10000, 10000 + args.phantoms), 1, int(args.low), int(args.high), rng_seed=1)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = gdrr.Cnn(max(64, args.batch), H, W, args.channels, seed=1)
    t0 = time.perf_counter()
    losses = train(net, X, Y, args.steps, args.batch, args.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = evaluate(net, n_low=int(args.low))
    res.update({"train_pairs": args.phantoms, "train_steps": args.steps, "channels": args.channels,
                "data_s": t_data, "train_s": t_train,
                "final_loss": float(np.mean(losses[-50:])), "input_histories": args.low,
                "target_histories": args.high})
    res["plain"] = {f"{n:.0e}": v for n, v in res["plain"].items()}
    print(json.dumps(res))
    net.close()


if __name__ == "__main__":
    main()
