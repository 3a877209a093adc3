"""Training of the learned band's encoder (dtw_encoder_grad, dtw_encoder_adam).

The encoder (include/pardtw.h, "learned band") is trained on exact
alignments of synthetic warped pairs: the exact DTW of every training pair
(dtw_align_many, the library's own exact path) gives, per coarse row of A,
the coarse column the embedding loss pulls the row's embedding towards
(mode 0); with the trunk trained, the half-width head is fitted to the band
each row needs around the coarse alignment of the learned embeddings
(mode 1).  The forward and backward passes and the optimiser step are the
library's kernels; this module only draws the data, orders the calls and
stores the parameters.

    python -m paper_2607_15478_gb300.band_train [--pairs 2000] [--epochs 3]
        [--out paper_2607_15478_gb300/weights/band_encoder_d12.npy]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(PKG, "weights", "band_encoder_d12.npy")


def layout(D: int):
    """Offsets (start, shape) of the parameter blocks in the flat array, in
    the order include/pardtw.h gives."""
    C, E, K = 64, 16, 5
    shapes = [("W1", (C, D, K)), ("b1", (C,)), ("W2", (C, C, K)), ("b2", (C,)),
              ("W3", (C, C, K)), ("b3", (C,)), ("W4", (E, C)), ("b4", (E,)),
              ("W5", (C,)), ("b5", (1,))]
    out, o = {}, 0
    for name, shp in shapes:
        out[name] = (o, shp)
        o += int(np.prod(shp))
    return out, o


def init_params(D: int, seed: int = 0) -> np.ndarray:
    """He-uniform weights for the ReLU layers, Glorot-uniform for the heads,
    zero biases except b5 = -2 (half-widths start near the smallest one)."""
    rng = np.random.default_rng(seed)
    lay, n = layout(D)
    p = np.zeros(n, dtype=np.float32)
    for name, (o, shp) in lay.items():
        size = int(np.prod(shp))
        if name in ("W1", "W2", "W3"):
            fan_in = shp[1] * shp[2]
            lim = math.sqrt(6.0 / fan_in)
        elif name == "W4":
            lim = math.sqrt(6.0 / (shp[0] + shp[1]))
        elif name == "W5":
            lim = math.sqrt(6.0 / (shp[0] + 1))
        else:
            continue
        p[o:o + size] = rng.uniform(-lim, lim, size=size).astype(np.float32)
    p[lay["b5"][0]] = -2.0
    return p


def exact_paths(al, As, Bs, chunk: int = 64):
    """Exact alignments of the pairs (device tensors) in chunks of dtw_align_many."""
    import torch
    paths, lens = [], []
    for c0 in range(0, len(As), chunk):
        ps, costs, st = al.align_many(As[c0:c0 + chunk], Bs[c0:c0 + chunk])
        if not (st == 0).all():
            raise RuntimeError(f"exact alignment failed: statuses {st}")
        for p in ps:
            paths.append(p.contiguous())
            lens.append(torch.tensor([p.shape[0]], dtype=torch.int32, device=p.device))
    return paths, lens


def train(n_pairs: int = 2000, epochs: int = 3, width_epochs: int = 1, lr: float = 1e-3,
          lr_width: float = 1e-2, seed: int = 0, device: int = 0, log=print):
    import torch
    from . import build, pardtw, synth
    build.build()
    al = pardtw.Aligner(device)
    dev = torch.device("cuda", device)
    t0 = time.perf_counter()
    pairs = [synth.band_training_pair(k) for k in range(n_pairs)]
    As = [torch.from_numpy(p.A).to(dev) for p in pairs]
    Bs = [torch.from_numpy(p.B).to(dev) for p in pairs]
    t_gen = time.perf_counter() - t0
    paths, lens = exact_paths(al, As, Bs)
    torch.cuda.synchronize(dev)
    t_exact = time.perf_counter() - t0 - t_gen
    log(f"{n_pairs} pairs drawn in {t_gen:.1f} s, exact alignments in {t_exact:.1f} s")
    D = pairs[0].A.shape[1]
    P = torch.from_numpy(init_params(D, seed)).to(dev)
    G = torch.zeros_like(P)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    order_rng = np.random.default_rng(seed + 1)
    step = 0
    history = []
    for mode, n_ep, rate in ((0, epochs, lr), (1, width_epochs, lr_width)):
        if mode == 1:  # the width head alone: fresh optimiser state
            M.zero_()
            V.zero_()
            step = 0
        for ep in range(n_ep):
            loss.zero_()
            te = time.perf_counter()
            for k in order_rng.permutation(n_pairs):
                pardtw.dtw_encoder_grad(al.h, P, As[k], Bs[k], paths[k], lens[k], mode, G, loss)
                step += 1
                pardtw.dtw_encoder_adam(al.h, P, G, M, V, step, rate)
            mean = float(loss.item()) / n_pairs
            history.append({"mode": mode, "epoch": ep, "mean_loss": mean,
                            "seconds": time.perf_counter() - te})
            log(f"mode {mode} epoch {ep}: mean loss {mean:.4f} "
                f"({time.perf_counter() - te:.1f} s)")
    al.close()
    meta = {"pairs": n_pairs, "epochs": epochs, "width_epochs": width_epochs, "lr": lr,
            "lr_width": lr_width, "seed": seed, "D": D, "history": history,
            "data": "synth.band_training_pair(k), k < pairs"}
    return P.cpu().numpy(), meta


def save(params: np.ndarray, meta: dict, path: str = DEFAULT_WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, params.astype(np.float32))
    with open(os.path.splitext(path)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)


def load(path: str = DEFAULT_WEIGHTS, device=None):
    """The stored parameters as a float32 tensor on `device` (CUDA)."""
    import torch
    p = np.load(path).astype(np.float32)
    return torch.from_numpy(p).to(device if device is not None else "cuda")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--width-epochs", type=int, default=1)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args()
    params, meta = train(a.pairs, a.epochs, a.width_epochs, a.lr, seed=a.seed)
    save(params, meta, a.out)
    print(f"saved {params.size} parameters to {a.out}")


if __name__ == "__main__":
    main()
