"""Training set and training of the warm-start network, on the GPU.

Every computation runs in the CUDA library: labels come from the library's
own cold-start batched FCM (random Dirichlet U^0, as in Algorithm 1 step 2),
features from its histogram kernel, and training from its forward/backward/
Adam kernels. Python only generates the synthetic slices (in spawned worker
processes), moves arrays and picks, per slice, the start with the lowest J.

Random starts do not always end at the same fixed point: on about 45% of the
synthetic slices, four seeded Dirichlet starts reach two or more different
local minima of J (Eq. 1). A label taken from one random start is then a
random draw, which no network can predict. The label of a slice is instead the
sorted centers of the start, among ``STARTS``, that ends with the lowest J.
The same fact sets the acceptance rule of a warm-started slice (``accepted``):
its centers match the cold start's within 1e-4 relative, or it ends at a
fixed point whose J is no larger than the cold start's.

Command line (writes the model file the warm-start runs load):

    python -m paper_1601_00072_gb300.warmstart --n-train 60000 \
        --out paper_1601_00072_gb300/data/warmstart.fcmw
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart.fcmw")
TRAIN_OFFSET = 1_000_000      # training slices are keyed (4, 1_000_000 + i), disjoint from the batch
STARTS = 4                    # random starts per training slice
START_STRIDE = 1000           # start s draws its U0 with key (U0_FAMILY + s * START_STRIDE, i)
CENTER_TOL = 1e-4             # warm and cold centers agree: max |dv| / max(|v|, 1) <= 1e-4
J_SLACK = 1e-5                # relative slack on J (FP32 kernels resolve J to about 1e-7)


def u0_key(i, s=0):
    """Generator key of the initial memberships of slice i, start s."""
    import phantom
    return (phantom.U0_FAMILY + s * START_STRIDE, i)


def _gen_slice(i, starts=1):
    """Image and the initial memberships of each start of generator slice i
    (worker process)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import phantom
    sp, img, _ = phantom.batch_slice(i)
    x = img.reshape(-1)
    return i, sp.C, x, [phantom.dirichlet_u0(u0_key(i, s), sp.C, x.size) for s in range(starts)]


def slices_of(indices, starts=1, workers=None, chunk=256):
    """Yields lists of (index, C, x uint8, [U0 of each start]) for the
    generator slices, in order, generated in parallel by spawned processes
    (no CUDA in them)."""
    from functools import partial
    indices = list(indices)
    workers = workers or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(workers, mp_context=ctx) as ex:
        for s in range(0, len(indices), chunk):
            yield list(ex.map(partial(_gen_slice, starts=starts), indices[s:s + chunk], chunksize=8))


def labelled_set(fcm, indices, starts=STARTS, workers=None, chunk=256):
    """Features [n, 264], targets [n, 8] (sorted centers / 255 of the start
    with the lowest final J, zero beyond C), C [n] (int32), all CUDA tensors,
    and the iteration counts of start 0."""
    import torch
    from .fcm import Slice
    F, T, Cs, its = [], [], [], []
    for part in slices_of(indices, starts, workers, chunk):
        xs = [torch.from_numpy(x.astype(np.float32)).cuda() for _, _, x, _ in part]
        best = [None] * len(part)
        for s in range(starts):
            slices = [Slice(x=xs[k], C=C, U0=torch.from_numpy(u0s[s]).cuda())
                      for k, (_, C, _, u0s) in enumerate(part)]
            fcm.run_batched(slices)
            if s == 0:
                F.append(fcm.features(slices))
                its.extend(sl.iters for sl in slices)
            for k, sl in enumerate(slices):
                if sl.status >= 0 and (best[k] is None or sl.J < best[k][0]):
                    best[k] = (sl.J, torch.sort(sl.V)[0] / 255.0)
            del slices
        t = torch.zeros((len(part), 8), dtype=torch.float32, device="cuda")
        for k, (_, C, _, _) in enumerate(part):
            t[k, :C] = best[k][1]
        T.append(t)
        Cs.append(torch.tensor([C for _, C, _, _ in part], dtype=torch.int32, device="cuda"))
    return torch.cat(F), torch.cat(T), torch.cat(Cs), np.array(its)


def accepted(cold, warm):
    """Per slice, whether the warm-started run is accepted against the cold
    start: sorted centers within ``CENTER_TOL`` relative, or a final J no
    larger than the cold start's (relative slack ``J_SLACK``)."""
    out = []
    for c, w in zip(cold, warm):
        vc = np.sort(np.asarray(c.V64[:c.C], dtype=np.float64))
        vw = np.sort(np.asarray(w.V64[:w.C], dtype=np.float64))
        same = np.max(np.abs(vw - vc) / np.maximum(np.abs(vc), 1.0)) <= CENTER_TOL
        better = w.status >= 0 and w.J <= c.J * (1.0 + J_SLACK)
        out.append(bool(same or better))
    return np.array(out)


def train(fcm, feats, targets, Cs, epochs=200, batch=256, lr=2e-3, seed=0):
    """Fresh network, trained on the GPU; returns the last epoch's mean loss."""
    fcm.model_init(seed)
    return fcm.model_train(feats, targets, Cs, epochs=epochs, batch=batch, lr=lr, seed=seed)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n-train", type=int, default=60000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--starts", type=int, default=STARTS)
    ap.add_argument("--workers", type=int, default=None)
    ap.add_argument("--out", default=MODEL_PATH)
    args = ap.parse_args(argv)
    from . import _build
    _build.build()
    from .fcm import FCM
    fcm = FCM(0)
    t0 = time.time()
    F, T, Cs, its = labelled_set(fcm, range(TRAIN_OFFSET, TRAIN_OFFSET + args.n_train), args.starts, args.workers)
    t1 = time.time()
    loss = train(fcm, F, T, Cs, args.epochs, args.batch, args.lr, args.seed)
    t2 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    fcm.model_save(args.out)
    print(json.dumps({"n_train": args.n_train, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
                      "seed": args.seed, "starts": args.starts, "final_loss": loss, "mean_cold_iters": float(its.mean()),
                      "label_seconds": round(t1 - t0, 1), "train_seconds": round(t2 - t1, 1),
                      "out": os.path.relpath(args.out, ROOT)}))


if __name__ == "__main__":
    main()
