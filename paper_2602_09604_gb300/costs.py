"""Algorithmic work of one fused-gate pass (used for roofline reporting and cost features).

Per group of 2^k amplitudes the complex mat-vec costs 2 * (3 * 4^k + 2^k * (2^k - 1)) flops:
4^k complex multiplies at 6 flops and 2^k * (2^k - 1) complex adds at 2 flops (section III gives
28 flops for k = 1; section IV-D gives the same numerator in its arithmetic-intensity formula).
Per amplitude that is 8 * 2^k - 2 flops.  A pass reads and writes every complex64 amplitude once:
16 bytes per amplitude.
"""
from __future__ import annotations


def flops_per_group(k: int) -> int:
    return 2 * (3 * 4 ** k + 2 ** k * (2 ** k - 1))


def flops_per_amp(k: int) -> float:
    return flops_per_group(k) / 2 ** k


def bytes_per_pass(n: int) -> int:
    return 16 * (1 << n)


def state_bytes(n: int) -> int:
    return 8 * (1 << n)


def ai_paper(f: int, num_vals: int) -> float:
    """Section IV-D's arithmetic intensity of the f-fused loop, as printed (numerator = flops per
    group, denominator numVals * 2^(f+3))."""
    return flops_per_group(f) / (num_vals * 2 ** (f + 3))
