"""Byte and flop counts of the paper's performance model (Sec. "Algorithm
Analysis and Optimization"): Table I, the traffic chain of Eq. 4, the
minimum code balance of Eqs. 5-7 and the roofline of Eq. 9.

S_d bytes per complex matrix/vector entry (16 for complex double, 8 for
complex float), S_i = 4 bytes per column index, F_a = 2 and F_m = 6 flops per
complex addition and multiplication.
"""
import math

S_I = 4
F_A = 2
F_M = 6


def sweep_bytes(n, nnz, R, sd, init=False):
    """Minimum bytes of one aug_spmmv sweep (one term of Eq. 4): the matrix
    once, V read, W read and written (the initial sweep does not read W)."""
    return nnz * (sd + S_I) + (2 if init else 3) * R * sd * n


def sweep_flops(n, nnz, R):
    """Flops of one sweep by Table I's count: R [N_nz (F_a + F_m) +
    N (ceil(7 F_a / 2) + ceil(9 F_m / 2))]."""
    return R * (nnz * (F_A + F_M) + n * (math.ceil(7 * F_A / 2) + math.ceil(9 * F_M / 2)))


def fused_fp64_flops(nnz, n, R, half=False):
    """Floating-point work the fused kernel executes with H' = 2a(H - b 1)
    folded: one complex multiply-add (8 flops) per stored entry and column,
    or 4 when every entry is purely real or purely imaginary (half=True: the
    other two products are zero), plus <V|V> and Re<W|V> (4 flops each) per
    row and column."""
    return R * ((4 if half else 8) * nnz + 8 * n)


def kpm_traffic(M, n, nnz, R, sd, variant="aug_spmmv"):
    """Eq. 4: minimum traffic of the whole solver for the naive algorithm
    (Fig. 3), aug_spmv (Fig. 4) and aug_spmmv (Fig. 5)."""
    if variant == "naive":
        return R * M / 2 * (nnz * (sd + S_I) + 13 * sd * n)
    if variant == "aug_spmv":
        return R * M / 2 * (nnz * (sd + S_I) + 3 * sd * n)
    if variant == "aug_spmmv":
        return M / 2 * (nnz * (sd + S_I) + 3 * R * sd * n)
    raise ValueError(variant)


def code_balance(nnzr, R, sd=16):
    """Minimum code balance B_min(R) in bytes/flop (Eq. 5 for the paper's
    values): (N_nzr/R (S_d + S_i) + 3 S_d) / (N_nzr (F_a + F_m) +
    ceil(7 F_a/2) + ceil(9 F_m/2))."""
    num = nnzr / R * (sd + S_I) + 3 * sd
    den = nnzr * (F_A + F_M) + math.ceil(7 * F_A / 2) + math.ceil(9 * F_M / 2)
    return num / den


def roofline(peak_flops, bandwidth, balance):
    """Eq. 9: P* = min(P_peak, b / B)."""
    return min(peak_flops, bandwidth / balance)
