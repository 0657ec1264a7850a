"""Train the residual post-filter (wv_cnn_*) on the GPU and write its
parameters.

Training pairs (--pairs, the shipped weights): a file of (decoded, original)
viewport luma pairs written by the oracle codec's pair generator
(oracle/filter_pairs.py): crops of seeded synthetic 8192 x 8192 frames coded
as YCbCr 4:2:0, 5-level CDF 9/7, one inter-frame Haar level, at one
dead-zone step, and projected into viewports with the same sampling as the
benchmark's 2160 x 2160, 110-degree viewports of 8192 frames, i.e. exactly
what the filtered decode feeds the network.  The last eighth of the
viewports (another crop) is held out.  Without --pairs: grey 2048 x 2048
frames coded and decoded by the library itself, whole-plane crops.

256 x 256 crops of (decoded, original) luma / 255 are the samples.  One
parameter set per step (the artefacts differ in strength; a single set
smooths low-distortion frames too much).  The network is trained with the
library's own forward/backward kernels (MSE, Adam).  The held-out set gives
the PSNR before and after.

    python -m oracle.filter_pairs --out /tmp/pairs --step 4
    python -m paper_2208_10859_gb300.train_postfilter --step 4 --pairs /tmp/pairs/pairs_q4.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
STEPS = (4.0, 6.0, 8.0, 12.0, 16.0)


def weights_path(step: float) -> str:
    """Parameter file of the network trained for quantiser step `step`."""
    return os.path.join(HERE, "weights", f"postfilter_q{int(step)}.bin")


def nearest_weights(step: float) -> str:
    return weights_path(min(STEPS, key=lambda s: abs(s - step)))


SIZE, PATCH = 2048, 256


def coded_pairs(wv, torch, seeds, steps, frames_per_seed=8):
    """Decoded and original luma (float32 / 255, on the device) per frame and step."""
    sys.path.insert(0, ROOT)
    import synth
    dec, org = [], []
    for seed in seeds:
        fr = synth.equirect_gop(SIZE, frames_per_seed, seed=seed, n_discs=30, chroma=False)
        dev = [tuple(torch.from_numpy(p).cuda() for p in f) for f in fr]
        for step in steps:
            desc = dict(width=SIZE, height=SIZE, planes=1, chroma_420=0, levels=5, wavelet=1,
                        num_frames=frames_per_seed, tlevels=0, block=256, quant=0, step=step)
            s = wv.Stream(wv.encode(dev, desc))
            for f in range(frames_per_seed):
                out = torch.empty((SIZE, SIZE), dtype=torch.uint8, device="cuda")
                s.decode_full(f, 0, out)
                dec.append(out.float() / 255)
                org.append(dev[f][0].float() / 255)
            torch.cuda.synchronize()
            s.close()
        del dev
    return torch.stack(dec), torch.stack(org)


def psnr(a, b) -> float:
    mse = float(((a - b) ** 2).mean())
    return 10 * math.log10(1.0 / mse)


def save_checkpoint(path: str, net, it: int, gen, log, torch) -> None:
    """Everything an interrupted run needs to continue exactly: parameters,
    Adam moments and step count, the iteration, the sampling generator's
    state and the loss log (a torch.save dict)."""
    m, v, k = net.state()
    torch.save({"params": net.params(), "adam_m": m, "adam_v": v, "adam_steps": k, "iteration": it,
                "rng": gen.get_state(), "log": list(log)}, path + ".tmp")
    os.replace(path + ".tmp", path)


def load_checkpoint(path: str, net, gen, torch):
    """Restore a checkpoint into net and gen; returns (iteration, log)."""
    ck = torch.load(path, weights_only=False)
    net.set_params(ck["params"])
    net.set_state(ck["adam_m"], ck["adam_v"], ck["adam_steps"])
    gen.set_state(ck["rng"])
    return int(ck["iteration"]), list(ck["log"])


def patch_pool(dec, n: int, patch: int, seed: int, torch):
    """The training set: n crops (frame, row, column) of patch x patch pairs,
    drawn once from the seed."""
    g = torch.Generator(device="cpu").manual_seed(seed + 7919)
    nfr, hh, ww = dec.shape
    return (torch.randint(0, nfr, (n,), generator=g), torch.randint(0, hh - patch + 1, (n,), generator=g),
            torch.randint(0, ww - patch + 1, (n,), generator=g))


def train(net, dec, org, pool, gen, steps: int, batch: int, patch: int, lr0: float, torch, start: int = 0,
          stop: int | None = None, log=None, checkpoint: str | None = None, every: int = 0,
          log_every: int = 200):
    """Adam on batches of the pool's patch pairs for iterations start .. stop - 1
    of a run of `steps` (cosine decay of the learning rate over the run);
    batches are drawn from gen.  Writes a checkpoint every `every` iterations
    and at the end when a path is given.  Returns the loss log [(iteration,
    loss)]."""
    log = [] if log is None else log
    stop = steps if stop is None else min(stop, steps)
    idx, ys, xs = pool
    for it in range(start, stop):
        sel = torch.randint(0, idx.shape[0], (batch,), generator=gen).tolist()
        xb = torch.stack([dec[idx[k], ys[k]:ys[k] + patch, xs[k]:xs[k] + patch] for k in sel])
        tb = torch.stack([org[idx[k], ys[k]:ys[k] + patch, xs[k]:xs[k] + patch] for k in sel])
        lr = lr0 * (0.5 * (1 + math.cos(math.pi * it / steps)) * 0.9 + 0.1)
        loss = net.train_step(xb.contiguous(), tb.contiguous(), lr, want_loss=(it % log_every == 0))
        if loss is not None:
            log.append((it, loss))
            print(f"step {it}/{steps} loss {loss:.3e}", flush=True)
        if checkpoint and every and (it + 1) % every == 0:
            save_checkpoint(checkpoint, net, it + 1, gen, log, torch)
    if checkpoint:
        save_checkpoint(checkpoint, net, stop, gen, log, torch)
    return log


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--step", type=float, required=True, choices=STEPS)
    ap.add_argument("--out", default=None)
    ap.add_argument("--patches", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--epochs", type=float, default=2.0)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--checkpoint", default=None, help="checkpoint file (written every --every iterations)")
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    ap.add_argument("--pairs", default=None, help="npz of (decoded, original) viewport luma pairs (dec, org)")
    args = ap.parse_args()
    import torch
    sys.path.insert(0, ROOT)
    from paper_2208_10859_gb300 import wv
    import __graft_entry__
    __graft_entry__.build()
    t0 = time.time()
    out = args.out or weights_path(args.step)
    if args.pairs:
        z = np.load(args.pairs)
        d = torch.from_numpy(z["dec"]).cuda().float() / 255
        o = torch.from_numpy(z["org"]).cuda().float() / 255
        hold = max(1, d.shape[0] // 8)
        dec, org, tdec, torg = d[:-hold], o[:-hold], d[-hold:], o[-hold:]
    else:
        dec, org = coded_pairs(wv, torch, (101, 102, 103, 104, 105, 106), (args.step,))
        tdec, torg = coded_pairs(wv, torch, (201,), (args.step,), frames_per_seed=4)
    g = torch.Generator(device="cpu").manual_seed(args.seed)
    net = wv.CNN(seed=args.seed)
    steps = int(args.epochs * args.patches / args.batch)
    pool = patch_pool(dec, args.patches, PATCH, args.seed, torch)
    start, log = 0, []
    if args.resume:
        start, log = load_checkpoint(args.checkpoint, net, g, torch)
    t1 = time.time()
    log = train(net, dec, org, pool, g, steps, args.batch, PATCH, args.lr, torch, start=start, log=log,
                checkpoint=args.checkpoint, every=args.every)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    if net.sync_status() != 0:
        raise RuntimeError("device error during training")
    # held-out PSNR
    x = tdec.contiguous()
    y = net.forward(x)
    y8 = torch.clamp(torch.floor(y * 255 + 0.5), 0, 255) / 255
    res = {"step": args.step, "decode_psnr": psnr(x, torg), "filtered_psnr": psnr(y8, torg)}
    p = net.params()
    os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
    p.astype("<f4").tofile(out)
    meta = {"pairs": os.path.basename(args.pairs) if args.pairs else "library codec, grey 2048^2 frames",
            "train_images": int(dec.shape[0]), "held_out_images": int(tdec.shape[0]),
            "patches": args.patches, "patch": PATCH, "batch": args.batch, "steps": steps, "lr": args.lr,
            "train_seconds": train_s, "total_seconds": time.time() - t0, "loss_log": log,
            "held_out_psnr": res, "params": int(p.size)}
    with open(os.path.splitext(out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
