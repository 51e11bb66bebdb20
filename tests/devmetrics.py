"""Fidelity and l2 distance between two device states in the library's blocked layout, in fp64,
computed on the device chunk by chunk (states of 30+ qubits do not fit on the host).

A state buffer is the torch tensor a ``DeviceState`` owns: blocks of 32 real then 32 imaginary
parts (fp32 for complex64 states, fp64 for complex128), so ``view(-1, 2, 32)`` gives
(block, re/im, lane) for either type.  Metrics as in the acceptance bar:
F = |<ref|psi>|^2 / (||ref||^2 ||psi||^2) and ||psi - ref||_2, both without phase alignment.
"""
from __future__ import annotations


def device_metrics(ref, psi, chunk_blocks: int = 1 << 21) -> dict:
    import torch
    a_all = ref.view(-1, 2, 32)
    b_all = psi.view(-1, 2, 32)
    assert a_all.shape == b_all.shape
    dev = ref.device
    ov = torch.zeros((), dtype=torch.complex128, device=dev)
    d2 = torch.zeros((), dtype=torch.float64, device=dev)
    na = torch.zeros((), dtype=torch.float64, device=dev)
    nb = torch.zeros((), dtype=torch.float64, device=dev)
    dmax = torch.zeros((), dtype=torch.float64, device=dev)
    for lo in range(0, a_all.shape[0], chunk_blocks):
        a = a_all[lo:lo + chunk_blocks].double()
        b = b_all[lo:lo + chunk_blocks].double()
        ca = torch.complex(a[:, 0], a[:, 1])
        cb = torch.complex(b[:, 0], b[:, 1])
        d = (cb - ca).abs()
        ov += (ca.conj() * cb).sum()
        d2 += (d * d).sum()
        na += (ca.abs() ** 2).sum()
        nb += (cb.abs() ** 2).sum()
        dmax = torch.maximum(dmax, d.max())
    return {"fidelity": float(ov.abs() ** 2 / (na * nb)), "l2_error": float(d2.sqrt()),
            "max_abs_error": float(dmax), "norm_ref": float(na), "norm": float(nb)}
