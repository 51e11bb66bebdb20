"""Device state buffers owned by PyTorch, wrapped as library states (marshalling only)."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class DeviceState:
    """A torch-allocated device buffer registered with sv_alloc (complex64) or sv_alloc_c128
    (complex128, c128=True) on a given CUDA stream."""

    def __init__(self, n: int, stream: torch.cuda.Stream | None = None, device: int | None = None, c128: bool = False):
        self.n = n
        self.c128 = bool(c128)
        self.nbytes = B.sv_required_bytes_c128(n) if self.c128 else B.sv_required_bytes(n)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        dt = torch.float64 if self.c128 else torch.float32
        self.buf = torch.empty(self.nbytes // dt.itemsize, dtype=dt, device=dev)
        alloc = B.sv_alloc_c128 if self.c128 else B.sv_alloc
        self.h = alloc(n, self.buf.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def init(self, basis_index: int = 0):
        B.sv_init(self.h, basis_index)

    def load(self, psi: np.ndarray):
        a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128 if self.c128 else np.complex64))
        assert a.size == (1 << self.n)
        B.sv_load(self.h, a.ctypes.data, True)
        self.stream.synchronize()   # the host array may be released after return

    def store(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex128 if self.c128 else np.complex64)
        B.sv_store(self.h, out.ctypes.data, True)
        return out

    def apply(self, fused, timings: bool = False):
        return B.sv_apply_fused_gates(self.h, fused, timings)

    def norm(self) -> float:
        return B.sv_norm(self.h)

    def sample(self, uniforms) -> np.ndarray:
        return B.sv_sample(self.h, uniforms)

    def expval(self, strings) -> np.ndarray:
        """<psi|P|psi> for Pauli strings given as {qubit: 'X' | 'Y' | 'Z'} dicts."""
        masks = [B.pauli_masks(t) for t in strings]
        return B.sv_expval_pauli(self.h, [m[0] for m in masks], [m[1] for m in masks])

    def free(self):
        if self.h is not None:
            B.sv_free(self.h)
            self.h = None
            self.buf = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
