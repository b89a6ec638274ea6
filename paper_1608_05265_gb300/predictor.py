"""Training data, training and evaluation of the learned predictors.

The library's autotuner times every legal configuration of a shape
(gbgemm_autotune); this module labels seeded sets of shapes with it, trains
the 3-layer MLP on the GPU through gbgemm_predictor_train (hand-written
forward/backward/Adam kernels), and measures the predictor's regret against
the tuner on held-out shapes.

    python -m paper_1608_05265_gb300.predictor --train 20000 --heldout 2000 \\
        --out paper_1608_05265_gb300/data/predictor_gb300.bin

The schedule predictor (tuning mode 2 of single calls) is trained the same
way on the schedule tuner's latencies (gbgemm_autotune_schedules, 39
schedules: path, tile, tile order and split-K slices):

    python -m paper_1608_05265_gb300.predictor --schedules --train 8000 --heldout 1000 \\
        --out paper_1608_05265_gb300/data/schedule_predictor_gb300.bin

Shape sets: m, n, k log-uniform integers in [8, 16384] (seed 4 for training,
seed 5 held out), transposes uniform over {N, T}, and a 16-byte alignment
class per operand (aligned: leading dimension a multiple of 4 and a 16-byte
aligned pointer; unaligned: an odd leading dimension).

Targets: y_c = log2(cost_c / min_c' cost_c') for every legal configuration c
(cost = the tuner's per-problem GPU time in a batch of copies; for schedules,
the latency of one call), masked elsewhere.
Regret of a choice c on a shape: cost_c / cost_best - 1.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import struct
import sys
import time

import numpy as np

from . import gbgemm, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "predictor_gb300.bin")
DEFAULT_SCHED_WEIGHTS = os.path.join(HERE, "data", "schedule_predictor_gb300.bin")
MAGIC = b"GBGEMM-MLP1\n"


def shape_set(seed: int, count: int, lo: int = 8, hi: int = 16384):
    """(ta, tb, m, n, k, align_a, align_b, align_c) tuples."""
    u = synth.draws(seed, 20, 3 * count)
    f = (u >> np.uint64(11)).astype(np.float64) * 2.0**-53
    dims = np.floor(np.exp(math.log(lo) + f * (math.log(hi + 1) - math.log(lo)))).astype(np.int64)
    dims = np.clip(dims, lo, hi).reshape(count, 3)
    fl = synth.draws(seed, 21, 5 * count).reshape(count, 5) >> np.uint64(63)
    out = []
    for g in range(count):
        out.append(("T" if fl[g, 0] else "N", "T" if fl[g, 1] else "N", int(dims[g, 0]), int(dims[g, 1]),
                    int(dims[g, 2]), int(fl[g, 2]), int(fl[g, 3]), int(fl[g, 4])))
    return out


def _ld(rows: int, aligned: int) -> int:
    if aligned:
        return (rows + 3) // 4 * 4
    return rows if rows % 2 == 1 else rows + 1


def tuning_problem(shape) -> gbgemm.Problem:
    """A problem descriptor carrying only what the tuner reads: shape, flags,
    leading dimensions and pointer alignment (the tuner times on its own
    buffers and never dereferences these addresses)."""
    ta, tb, m, n, k, aa, ab, ac = shape
    ar = m if ta == "N" else k
    br = k if tb == "N" else n
    lda, ldb, ldc = _ld(ar, aa), _ld(br, ab), _ld(m, ac)
    fake = lambda aligned: 0x10000 if aligned else 0x10004  # noqa: E731
    return gbgemm.problem(ta, tb, m, n, k, 1.0, fake(aa), lda, fake(ab), ldb, 0.0, fake(ac), ldc)


def features(shapes) -> np.ndarray:
    return np.array([gbgemm.predictor_features(tuning_problem(s)) for s in shapes], dtype=np.float32)


def label(handle: gbgemm.Handle, shapes, reps: int = 2, log_every: int = 0):
    """Tuner costs (n x 6, -1 illegal) and latencies of every shape."""
    cost = np.full((len(shapes), gbgemm.NUM_CONFIGS), -1.0, dtype=np.float64)
    lat = np.full_like(cost, -1.0)
    t0 = time.time()
    for i, s in enumerate(shapes):
        l, c, _, _ = handle.autotune(tuning_problem(s), reps=reps)
        lat[i] = l
        cost[i] = c
        if log_every and (i + 1) % log_every == 0:
            sys.stderr.write(f"labelled {i + 1}/{len(shapes)} in {time.time() - t0:.1f}s\n")
    return cost, lat


def label_schedules(handle: gbgemm.Handle, shapes, reps: int = 2, log_every: int = 0):
    """Schedule tuner latencies (n x 39, -1 illegal) of every shape."""
    lat = np.full((len(shapes), gbgemm.NUM_SCHEDULES), -1.0, dtype=np.float64)
    t0 = time.time()
    for i, s in enumerate(shapes):
        lat[i], _ = handle.autotune_schedules(tuning_problem(s), reps=reps)
        if log_every and (i + 1) % log_every == 0:
            sys.stderr.write(f"labelled {i + 1}/{len(shapes)} in {time.time() - t0:.1f}s\n")
    return lat


def default_schedules(handle: gbgemm.Handle, shapes) -> np.ndarray:
    """The library's fixed heuristic (tuning mode 0) for each shape."""
    return np.array([handle.schedule_default(tuning_problem(s)) for s in shapes], dtype=np.int64)


def legal_bytes(cost: np.ndarray) -> np.ndarray:
    """Legal masks, (n, ceil(C / 8)) bytes, bit c % 8 of byte c / 8 for output c."""
    nb = (cost.shape[1] + 7) // 8
    out = np.zeros((cost.shape[0], nb), dtype=np.uint8)
    for c in range(cost.shape[1]):
        out[:, c // 8] |= ((cost[:, c] > 0).astype(np.uint8) << (c % 8))
    return out


def targets(cost: np.ndarray):
    """(y, mask): log2(cost / best) on legal configurations."""
    mask = (cost > 0).astype(np.float32)
    safe = np.where(cost > 0, cost, np.inf)
    best = safe.min(axis=1, keepdims=True)
    y = np.where(cost > 0, np.log2(np.maximum(cost, 1e-9) / best), 0.0).astype(np.float32)
    return y, mask


def legal_bits(cost: np.ndarray) -> np.ndarray:
    bits = np.zeros(cost.shape[0], dtype=np.uint8)
    for c in range(cost.shape[1]):
        bits |= ((cost[:, c] > 0).astype(np.uint8) << c)
    return bits


def regret(cost: np.ndarray, choice: np.ndarray) -> dict:
    """Regret statistics of configuration choices against the per-shape best."""
    safe = np.where(cost > 0, cost, np.inf)
    best = safe.min(axis=1)
    chosen = cost[np.arange(len(choice)), choice]
    ratio = chosen / best
    r = ratio - 1.0
    return {"mean": float(r.mean()), "geomean_ratio": float(np.exp(np.log(ratio).mean())),
            "p95": float(np.percentile(r, 95)), "max": float(r.max()), "exact": float((r == 0).mean())}


def default_choice(shapes) -> np.ndarray:
    """The library's fixed heuristic (GBGEMM_CONFIG_DEFAULT) for each shape."""
    out = []
    for (ta, tb, m, n, k, *_rest) in shapes:
        if k >= 16:
            out.append(gbgemm.CFG_SPLIT_BN64 if n <= 64 else gbgemm.CFG_SPLIT_BN128)
        else:
            out.append(gbgemm.CFG_SIMT_128x128)
    return np.array(out, dtype=np.int64)


def save_weights(path: str, params: np.ndarray, meta: dict):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    head = json.dumps(dict(meta, format="gbgemm-mlp-v1", params=int(params.size), dtype="float32-le")).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(head)))
        f.write(head)
        f.write(np.ascontiguousarray(params, dtype="<f4").tobytes())


def load_weights(path: str = DEFAULT_WEIGHTS, n_params: int = gbgemm.MLP_PARAMS):
    with open(path, "rb") as f:
        if f.read(len(MAGIC)) != MAGIC:
            raise ValueError(f"{path}: not a predictor weights file")
        (n,) = struct.unpack("<I", f.read(4))
        meta = json.loads(f.read(n).decode())
        params = np.frombuffer(f.read(), dtype="<f4").astype(np.float32)
    if params.size != n_params or meta.get("params") != n_params:
        raise ValueError(f"{path}: expected {n_params} parameters")
    return params, meta


def train(handle: gbgemm.Handle, X: np.ndarray, y: np.ndarray, mask: np.ndarray, epochs: int, batch: int = 256,
          lr: float = 2e-3, seed: int = 4) -> float:
    import torch
    dx = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    dy = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).cuda()
    dm = torch.from_numpy(np.ascontiguousarray(mask, dtype=np.float32)).cuda()
    return handle.predictor_train(dx, dy, dm, epochs=epochs, batch=batch, lr=lr, seed=seed)


def predict(handle: gbgemm.Handle, X: np.ndarray, legal: np.ndarray, n_out: int = gbgemm.NUM_CONFIGS):
    import torch
    dx = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    dl = torch.from_numpy(np.ascontiguousarray(legal, dtype=np.uint8)).cuda()
    scores = torch.empty((X.shape[0], n_out), dtype=torch.float32, device="cuda")
    cfg = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    handle.predictor_predict(dx, dl, scores, cfg)
    torch.cuda.synchronize()
    return cfg.cpu().numpy().astype(np.int64), scores.cpu().numpy()


def main(argv=None):
    ap = argparse.ArgumentParser(description="label, train and evaluate the configuration predictor")
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=2000)
    ap.add_argument("--train-seed", type=int, default=4)
    ap.add_argument("--heldout-seed", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default=None, help="write a JSON report here")
    ap.add_argument("--cache", default=None, help="tuning cache file to resume from and update")
    ap.add_argument("--schedules", action="store_true", help="the single-call schedule predictor")
    ap.add_argument("--dump", default=None, help="save the shapes' labels here (.npz)")
    args = ap.parse_args(argv)
    if args.schedules:
        return main_schedules(args)
    import torch
    h = gbgemm.Handle(0)
    h.set_stream(torch.cuda.current_stream())
    if args.cache and os.path.exists(args.cache):
        h.tuning_load(args.cache)
    tr = shape_set(args.train_seed, args.train)
    ho = shape_set(args.heldout_seed, args.heldout)
    t0 = time.time()
    c_tr, _ = label(h, tr, reps=args.reps, log_every=1000)
    c_ho, _ = label(h, ho, reps=args.reps)
    t_label = time.time() - t0
    if args.cache:
        h.tuning_save(args.cache)
    X_tr, X_ho = features(tr), features(ho)
    y_tr, m_tr = targets(c_tr)
    t0 = time.time()
    loss = train(h, X_tr, y_tr, m_tr, epochs=args.epochs, seed=args.train_seed)
    t_train = time.time() - t0
    y_ho, m_ho = targets(c_ho)
    choice, scores = predict(h, X_ho, legal_bits(c_ho))
    ho_loss = float((((scores - y_ho) * m_ho) ** 2).sum() / m_ho.sum())
    rep = {"train_shapes": len(tr), "heldout_shapes": len(ho), "label_seconds": t_label, "train_seconds": t_train,
           "train_loss": loss, "heldout_loss": ho_loss,
           "regret_predictor": regret(c_ho, choice), "regret_default": regret(c_ho, default_choice(ho))}
    params = h.predictor_get()
    save_weights(args.out, params, {"train_seed": args.train_seed, "train_shapes": len(tr), "epochs": args.epochs,
                                    "train_loss": loss, "heldout_loss": ho_loss})
    print(json.dumps(rep, indent=1))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)
    h.close()


def main_schedules(args):
    """Label, train and evaluate the schedule predictor (network 1)."""
    import torch
    h = gbgemm.Handle(0)
    h.set_stream(torch.cuda.current_stream())
    if args.cache and os.path.exists(args.cache):
        h.tuning_load(args.cache)
    tr = shape_set(args.train_seed, args.train)
    ho = shape_set(args.heldout_seed, args.heldout)
    t0 = time.time()
    c_tr = label_schedules(h, tr, reps=args.reps, log_every=1000)
    c_ho = label_schedules(h, ho, reps=args.reps)
    t_label = time.time() - t0
    if args.dump:
        np.savez(args.dump, train=c_tr, heldout=c_ho, default_train=default_schedules(h, tr),
                 default_heldout=default_schedules(h, ho), x_train=features(tr), x_heldout=features(ho))
    if args.cache:
        h.tuning_save(args.cache)
    h.predictor_select(1)
    X_tr, X_ho = features(tr), features(ho)
    y_tr, m_tr = targets(c_tr)
    t0 = time.time()
    loss = train(h, X_tr, y_tr, m_tr, epochs=args.epochs, seed=args.train_seed)
    t_train = time.time() - t0
    y_ho, m_ho = targets(c_ho)
    choice, scores = predict(h, X_ho, legal_bytes(c_ho), gbgemm.NUM_SCHEDULES)
    ho_loss = float((((scores - y_ho) * m_ho) ** 2).sum() / m_ho.sum())
    rep = {"network": "schedules", "train_shapes": len(tr), "heldout_shapes": len(ho), "label_seconds": t_label,
           "train_seconds": t_train, "train_loss": loss, "heldout_loss": ho_loss,
           "legal_per_shape": float((c_ho > 0).sum(1).mean()),
           "regret_predictor": regret(c_ho, choice), "regret_default": regret(c_ho, default_schedules(h, ho))}
    params = h.predictor_get()
    out = args.out if args.out != DEFAULT_WEIGHTS else DEFAULT_SCHED_WEIGHTS
    save_weights(out, params, {"network": "schedules", "train_seed": args.train_seed, "train_shapes": len(tr),
                               "epochs": args.epochs, "train_loss": loss, "heldout_loss": ho_loss})
    print(json.dumps(rep, indent=1))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rep, f, indent=1)
    h.close()


if __name__ == "__main__":
    main()
