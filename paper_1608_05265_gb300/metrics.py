"""FLOP and byte counting for sgemm throughput figures.

Throughput follows the paper's convention (Section IV, Tables I-VI):
GFLOPS = 2*m*n*K / seconds; the beta*C update is not counted.
"""


def gemm_flops(m: int, n: int, k: int) -> float:
    """Algorithmic FLOPs of one sgemm: one multiply and one add per (i, j, p)."""
    return 2.0 * float(m) * float(n) * float(k)


def gemm_min_bytes(m: int, n: int, k: int, beta_reads_c: bool = True) -> float:
    """Compulsory HBM bytes of one FP32 sgemm: read A, B (and C), write C."""
    c_rw = 2 if beta_reads_c else 1
    return 4.0 * (float(m) * k + float(k) * n + c_rw * float(m) * n)


def split_pack_bytes(rows: int, k: int) -> float:
    """Algorithmic bytes of the split-and-pack step for one operand.

    One read of the FP32 operand for the row maxima, one read to split it and
    one write of the hi/lo BF16 panel (2 x 2 bytes per element, k rounded up
    to the 32-element chunk).
    """
    kp = (k + 31) // 32 * 32
    return 4.0 * rows * k * 2 + 4.0 * rows * kp
