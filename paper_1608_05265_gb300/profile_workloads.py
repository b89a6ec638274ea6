"""Fixed workloads for profiling the library under ncu (one GPU).

    python -m paper_1608_05265_gb300.profile_workloads <name> [--reps R]

runs one workload R times on cuda:0 through the C-ABI binding and exits 0.
Inputs are seeded and generated on the device; nothing is timed or printed
beyond a one-line summary.  Names:

  split4096   sgemm 4096^3 NN, ld 4104, split path (alpha 1.5, beta -0.25)
  simt4096    the same on the FP32 SIMT path
  split8192   sgemm 8192^3 NN, ld 8200, split path (the headline shape)
  split1024 / split2048 / simt8192
              the same shape family at n = 1024 and 2048 (split path), and
              8192 on the SIMT path
  grouped     the uneven batch (m, n, k log-uniform in [16, 1024], seed 3;
              4096 problems, or --count), one plan with the default
              configurations
  linpack8192 / linpack16384
              the Linpack-shaped update C(m x m) -= A(m x 128) B(128 x m),
              normal entries, split path
  gemv        sgemv with A 16384 x 16384 (1.07 GB), op(A) = A then A^T
  splitk      512 x 512 x 65536 on the split path (k sliced, then reduced)
  mlp         the predictor: 20 epochs of training on 4096 synthetic rows,
              then inference on 4096 rows
  lu4608      sgetrf + sgetrs, N 4608 (the paper's HPL size), default block
"""

from __future__ import annotations

import argparse


def _split_or_simt(h, path, reps, n=4096):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    ld = n + 8
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.rand(ld * n, device="cuda", generator=g) * 2 - 1
    B = torch.rand(ld * n, device="cuda", generator=g) * 2 - 1
    C = torch.rand(ld * n, device="cuda", generator=g) * 2 - 1
    h.set_path(gbgemm.PATH_SPLIT_BF16 if path == "split" else gbgemm.PATH_SIMT)
    for _ in range(reps):
        h.sgemm("N", "N", n, n, n, 1.5, A, ld, B, ld, -0.25, C, ld)
    torch.cuda.synchronize()


def _grouped(h, reps, count=4096):
    import torch
    from paper_1608_05265_gb300 import gbgemm, synth
    shapes = synth.grouped_shapes(3, count)
    g = torch.Generator(device="cuda").manual_seed(3)
    bufs, probs = [], []
    for (ta, tb, m, n, k) in shapes:
        ar, ac = synth.op_shape(ta, m, k)
        br, bc = synth.op_shape(tb, k, n)
        A = torch.rand(ar * ac, device="cuda", generator=g) * 2 - 1
        B = torch.rand(br * bc, device="cuda", generator=g) * 2 - 1
        C = torch.empty(m * n, device="cuda")
        bufs.append((A, B, C))
        probs.append(gbgemm.problem(ta, tb, m, n, k, 1.0, A, ar, B, br, 0.0, C, m))
    plan = gbgemm.GroupedPlan(h, probs, config_source=gbgemm.CONFIG_DEFAULT)
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        plan.run(stream)
    torch.cuda.synchronize()
    plan.close()


def _linpack(h, reps, m, nb=128):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    g = torch.Generator(device="cuda").manual_seed(20 + nb)
    A = torch.randn(m * nb, device="cuda", generator=g)
    B = torch.randn(nb * m, device="cuda", generator=g)
    C = torch.randn(m * m, device="cuda", generator=g)
    h.set_path(gbgemm.PATH_AUTO)
    for _ in range(reps):
        h.sgemm("N", "N", m, m, nb, -1.0, A, m, B, nb, 1.0, C, m)
    torch.cuda.synchronize()


def _gemv(h, reps, n=16384):
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.rand(n * n, device="cuda", generator=g) * 2 - 1
    x = torch.rand(n, device="cuda", generator=g) * 2 - 1
    y = torch.zeros(n, device="cuda")
    for _ in range(reps):
        h.sgemv("N", n, n, 1.0, A, n, x, 1, 0.0, y, 1)
        h.sgemv("T", n, n, 1.0, A, n, x, 1, 0.0, y, 1)
    torch.cuda.synchronize()


def _splitk(h, reps):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    m = n = 512
    k = 65536
    g = torch.Generator(device="cuda").manual_seed(6)
    A = torch.rand(m * k, device="cuda", generator=g) * 2 - 1
    B = torch.rand(k * n, device="cuda", generator=g) * 2 - 1
    C = torch.zeros(m * n, device="cuda")
    h.set_path(gbgemm.PATH_SPLIT_BF16)
    for _ in range(reps):
        h.sgemm("N", "N", m, n, k, 1.0, A, m, B, k, 0.0, C, m)
    torch.cuda.synchronize()


def _mlp(h, reps):
    import numpy as np
    import torch
    from paper_1608_05265_gb300 import gbgemm
    rng = np.random.default_rng(9)
    X = torch.from_numpy(rng.uniform(0, 1, (4096, 8)).astype(np.float32)).cuda()
    Y = torch.from_numpy(rng.uniform(0, 1, (4096, gbgemm.NUM_CONFIGS)).astype(np.float32)).cuda()
    M = torch.ones_like(Y)
    legal = torch.full((4096,), (1 << gbgemm.NUM_CONFIGS) - 1, dtype=torch.uint8, device="cuda")
    scores = torch.empty_like(Y)
    cfg = torch.empty(4096, dtype=torch.int32, device="cuda")
    for _ in range(reps):
        h.predictor_train(X, Y, M, epochs=20, batch=256, lr=1e-3, seed=1)
        h.predictor_predict(X, legal, scores, cfg)
    torch.cuda.synchronize()


def _lu(h, reps):
    import torch
    n = 4608
    g = torch.Generator(device="cuda").manual_seed(8)
    A0 = torch.rand(n * n, device="cuda", generator=g) - 0.5
    b0 = torch.rand(n, device="cuda", generator=g) - 0.5
    piv = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.empty(1, dtype=torch.int32, device="cuda")
    for _ in range(reps):
        A, b = A0.clone(), b0.clone()
        h.sgetrf(n, A, n, piv, info)
        h.sgetrs(n, 1, A, n, piv, b, n)
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError(f"sgetrf info {int(info.item())}")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["split1024", "split2048", "split4096", "simt4096", "split8192", "simt8192",
                                     "grouped", "lu4608", "linpack8192", "linpack16384", "gemv", "splitk", "mlp"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--count", type=int, default=4096, help="problems of the grouped batch")
    args = ap.parse_args(argv)
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    h = gbgemm.Handle(0)
    h.set_stream(torch.cuda.current_stream())
    if args.name in ("split1024", "split2048", "split4096", "simt4096", "split8192", "simt8192"):
        _split_or_simt(h, args.name[:-4], args.reps, int(args.name[-4:]))
    elif args.name == "grouped":
        _grouped(h, args.reps, args.count)
    elif args.name.startswith("linpack"):
        _linpack(h, args.reps, int(args.name[len("linpack"):]))
    elif args.name == "gemv":
        _gemv(h, args.reps)
    elif args.name == "splitk":
        _splitk(h, args.reps)
    elif args.name == "mlp":
        _mlp(h, args.reps)
    else:
        _lu(h, args.reps)
    status = h.get_device_status()
    h.close()
    print(f"{args.name}: {args.reps} runs, device status {status}")
    return 0 if status == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
