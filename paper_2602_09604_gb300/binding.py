"""Thin ctypes binding of libsvgb300.so (the C ABI declared in include/sv_gb300.h).

Argument marshalling only: every step of the simulation runs inside the library.  The functions
keep the C names.  Failures raise :class:`SvError` carrying the library's status code and message.
There is deliberately no fallback: if the library has not been built (``__graft_entry__.build()``
or ``python -m paper_2602_09604_gb300.build``) importing this module raises.
"""
from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsvgb300.so")

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ETIMEOUT, SV_EUNITARY, SV_ESTATE = 0, -1, -2, -3, -4, -5, -6
PATH_AUTO, PATH_LOW, PATH_HIGH, PATH_MIXED, PATH_TC_TF32, PATH_TC_BF16X3, PATH_CONTROLLED, PATH_SWAPS = range(8)
PATH_NAMES = {PATH_AUTO: "auto", PATH_LOW: "low", PATH_HIGH: "high", PATH_MIXED: "mixed",
              PATH_TC_TF32: "tc_tf32", PATH_TC_BF16X3: "tc_bf16x3", PATH_CONTROLLED: "controlled",
              PATH_SWAPS: "swaps"}
PATH_POST_PHASES = 256   # flag or-ed into the path a cost function sees for a gate with post-phases
PREC_FP32, PREC_TF32, PREC_BF16X3 = 0, 1, 2
FUSE_GREEDY, FUSE_LEARNED, FUSE_NONE, FUSE_PHASES = 0, 1, 2, 3
MAX_K = 6
MAX_CONTROLS = 33


class SvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class sv_gate(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("targets", ctypes.c_int * MAX_K), ("n_controls", ctypes.c_int),
                ("controls", ctypes.c_int * MAX_CONTROLS), ("mat", ctypes.POINTER(ctypes.c_double))]


COST_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p)


class sv_fuse_opts(ctypes.Structure):
    _fields_ = [("max_k", ctypes.c_int), ("mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("tc_min_k", ctypes.c_int), ("force_path", ctypes.c_int), ("model", ctypes.c_void_p),
                ("start_qubits", ctypes.c_int), ("cost_us", COST_FN), ("cost_ctx", ctypes.c_void_p)]


class sv_fused_info(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("targets", ctypes.c_int * MAX_K), ("path", ctypes.c_int),
                ("n_source_gates", ctypes.c_int), ("control_mask", ctypes.c_uint64)]


class sv_mlp_train_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("val_frac", ctypes.c_float), ("fallback_k", ctypes.c_int)]


class sv_mlp_stats(ctypes.Structure):
    _fields_ = [("train_loss", ctypes.c_float), ("val_mape", ctypes.c_float), ("n_train", ctypes.c_longlong),
                ("n_val", ctypes.c_longlong), ("steps", ctypes.c_longlong), ("trained", ctypes.c_int),
                ("y_mean", ctypes.c_float), ("y_std", ctypes.c_float), ("fallback_k", ctypes.c_int)]


class sv_batch_opts(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("smem_max_n", ctypes.c_int), ("ctas", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("split_min_n", ctypes.c_int), ("tile_log2", ctypes.c_int),
                ("wave_mb", ctypes.c_int), ("stage_log2", ctypes.c_int), ("stage_k", ctypes.c_int),
                ("stage_layers", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class sv_batch_info(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int), ("whole", ctypes.c_int), ("single", ctypes.c_int), ("split", ctypes.c_int),
                ("staged", ctypes.c_int), ("stages", ctypes.c_int), ("stage_gates", ctypes.c_int),
                ("traffic_bytes", ctypes.c_double)]


TIMING_SMALL_SOURCE = 1   # sv_timing.flags: inputs read from the lazy start's small state


class sv_timing(ctypes.Structure):
    _fields_ = [("us", ctypes.c_float), ("k", ctypes.c_int), ("path", ctypes.c_int), ("flags", ctypes.c_int),
                ("target_mask", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -m paper_2602_09604_gb300.build); there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    sig = {
        "sv_required_bytes": (ctypes.c_size_t, [I]),
        "sv_alloc": (I, [I, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "sv_required_bytes_c128": (ctypes.c_size_t, [I]),
        "sv_alloc_c128": (I, [I, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "sv_free": (None, [P]),
        "sv_init": (I, [P, ctypes.c_uint64]),
        "sv_load": (I, [P, P, I]),
        "sv_store": (I, [P, P, I]),
        "sv_fuse_circuit": (I, [ctypes.POINTER(sv_gate), I, I, ctypes.POINTER(sv_fuse_opts), ctypes.POINTER(P)]),
        "sv_fused_free": (None, [P]),
        "sv_fused_count": (I, [P]),
        "sv_fused_get_info": (I, [P, I, ctypes.POINTER(sv_fused_info)]),
        "sv_fused_get_matrix": (I, [P, I, ctypes.POINTER(ctypes.c_double)]),
        "sv_fused_get_post_phases": (I, [P, I, I, P, P, P]),
        "sv_fused_get_swaps": (I, [P, I, I, P, P]),
        "sv_apply_fused_gates": (I, [P, P, ctypes.POINTER(sv_timing)]),
        "sv_init_apply": (I, [P, ctypes.c_uint64, P, ctypes.POINTER(sv_timing)]),
        "sv_norm": (I, [P, ctypes.POINTER(ctypes.c_double)]),
        "sv_sample": (I, [P, ctypes.POINTER(ctypes.c_double), I, ctypes.POINTER(ctypes.c_uint64)]),
        "sv_sample_norm": (I, [P, ctypes.POINTER(ctypes.c_double), I, ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_double)]),
        "sv_sample_noalloc": (I, [P, I, P, ctypes.POINTER(ctypes.c_double), I, ctypes.POINTER(ctypes.c_uint64)]),
        "sv_device_status": (I, []),
        "sv_expval_pauli": (I, [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), I,
                                ctypes.POINTER(ctypes.c_double)]),
        "sv_batch_arena_bytes": (ctypes.c_size_t, [ctypes.POINTER(ctypes.c_int), I]),
        "sv_batch_create": (I, [ctypes.POINTER(P), I, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "sv_batch_free": (None, [P]),
        "sv_batch_set_opts": (I, [P, ctypes.POINTER(sv_batch_opts)]),
        "sv_batch_get_opts": (I, [P, ctypes.POINTER(sv_batch_opts)]),
        "sv_batch_run": (I, [P]),
        "sv_batch_run_loop": (I, [P]),
        "sv_batch_state_offset": (I, [P, I, ctypes.POINTER(ctypes.c_size_t)]),
        "sv_batch_plan_stages": (I, [P, I, I, P, P, P, P, P]),
        "sv_batch_inject_stall": (I, [P, I]),
        "sv_batch_get_info": (I, [P, ctypes.POINTER(sv_batch_info)]),
        "sv_mlp_num_params": (I, []),
        "sv_mlp_create": (I, [ctypes.c_uint64, P, ctypes.POINTER(P)]),
        "sv_mlp_free": (None, [P]),
        "sv_mlp_get_params": (I, [P, ctypes.POINTER(ctypes.c_float)]),
        "sv_mlp_set_params": (I, [P, ctypes.POINTER(ctypes.c_float)]),
        "sv_mlp_features": (I, [I, ctypes.POINTER(ctypes.c_int), I, I, I, ctypes.POINTER(ctypes.c_float)]),
        "sv_mlp_gradients": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), I,
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "sv_mlp_adam_step": (I, [P, ctypes.c_float]),
        "sv_mlp_train": (I, [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_longlong,
                             ctypes.POINTER(sv_mlp_train_opts), ctypes.POINTER(sv_mlp_stats)]),
        "sv_mlp_predict": (I, [P, ctypes.POINTER(ctypes.c_float), I, ctypes.POINTER(ctypes.c_double)]),
        "sv_mlp_get_stats": (I, [P, ctypes.POINTER(sv_mlp_stats)]),
        "sv_mlp_save": (I, [P, ctypes.c_char_p]),
        "sv_mlp_load": (I, [ctypes.c_char_p, P, ctypes.POINTER(P)]),
        "sv_last_error": (ctypes.c_char_p, []),
        "sv_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def sv_last_error() -> str:
    return lib.sv_last_error().decode()


def _check(rc: int):
    if rc != SV_OK:
        raise SvError(rc, sv_last_error())


# --------------------------------------------------------------------------------------- state
def sv_required_bytes(n: int) -> int:
    return int(lib.sv_required_bytes(n))


def sv_alloc(n: int, dev_ptr: int, nbytes: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib.sv_alloc(n, ctypes.c_void_p(dev_ptr), nbytes, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def sv_required_bytes_c128(n: int) -> int:
    return int(lib.sv_required_bytes_c128(n))


def sv_alloc_c128(n: int, dev_ptr: int, nbytes: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib.sv_alloc_c128(n, ctypes.c_void_p(dev_ptr), nbytes, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def sv_free(h) -> None:
    lib.sv_free(h)


def sv_init(h, basis_index: int = 0) -> None:
    _check(lib.sv_init(h, ctypes.c_uint64(basis_index)))


def sv_load(h, src_ptr: int, on_host: bool) -> None:
    _check(lib.sv_load(h, ctypes.c_void_p(src_ptr), int(bool(on_host))))


def sv_store(h, dst_ptr: int, on_host: bool) -> None:
    _check(lib.sv_store(h, ctypes.c_void_p(dst_ptr), int(bool(on_host))))


# --------------------------------------------------------------------------------------- fusion
_GATE_DTYPE = np.dtype({"names": ["k", "targets", "n_controls", "controls", "mat"],
                        "formats": [np.int32, (np.int32, MAX_K), np.int32, (np.int32, MAX_CONTROLS), np.uint64],
                        "offsets": [sv_gate.k.offset, sv_gate.targets.offset, sv_gate.n_controls.offset,
                                    sv_gate.controls.offset, sv_gate.mat.offset],
                        "itemsize": ctypes.sizeof(sv_gate)})


def gate_array(gates):
    """sv_gate records for gate objects with .targets/.controls/.matrix, built as one numpy
    structured array laid out like the C struct (matrices packed into one complex128 buffer);
    returns (pointer to the records, keepalive) -- keep both alive for the duration of the call."""
    gates = list(gates)
    n = len(gates)
    rec = np.zeros(max(n, 1), dtype=_GATE_DTYPE)
    if n == 0:
        buf = np.zeros(1, dtype=np.complex128)
        return rec.ctypes.data_as(ctypes.POINTER(sv_gate)), (rec, buf)
    tl = [g.targets for g in gates]
    cl = [g.controls for g in gates]
    ks = np.fromiter(map(len, tl), dtype=np.int32, count=n)
    ncs = np.fromiter(map(len, cl), dtype=np.int32, count=n)
    bad = np.flatnonzero((ks > MAX_K) | (ncs > MAX_CONTROLS))
    if bad.size:
        raise SvError(SV_EINVAL, f"gate {int(bad[0])}: sv_gate holds at most {MAX_K} targets and {MAX_CONTROLS} controls")

    def scatter(field, lists, counts):
        total = int(counts.sum())
        if total == 0:
            return
        flat = np.fromiter(itertools.chain.from_iterable(lists), dtype=np.int32, count=total)
        starts = np.repeat(np.cumsum(counts) - counts, counts)
        rec[field][np.repeat(np.arange(n), counts), np.arange(total) - starts] = flat

    rec["k"][:n] = ks
    rec["n_controls"][:n] = ncs
    scatter("targets", tl, ks)
    scatter("controls", cl, ncs)
    mats = [np.asarray(g.matrix, dtype=np.complex128).reshape(-1) for g in gates]
    buf = np.concatenate(mats)
    sizes = np.fromiter((m.size for m in mats), dtype=np.uint64, count=n)
    offs = np.cumsum(sizes) - sizes
    rec["mat"][:n] = np.uint64(buf.ctypes.data) + np.uint64(16) * offs
    return rec.ctypes.data_as(ctypes.POINTER(sv_gate)), (rec, buf)


def sv_fuse_circuit(gates, n: int, max_k: int = 4, mode: int = FUSE_GREEDY, precision: int = PREC_FP32,
                    tc_min_k: int = 5, force_path: int = PATH_AUTO, model=None, start_qubits: int = 0,
                    cost_fn=None) -> ctypes.c_void_p:
    """cost_fn (learned mode, instead of a model): cost_fn(k, targets tuple, path, n) -> microseconds."""
    gl = list(gates)
    arr, keep = gate_array(gl)
    cb = COST_FN(lambda k, t, p, nq, ctx: float(cost_fn(k, tuple(t[i] for i in range(k)), p, nq))) if cost_fn else COST_FN()
    opts = sv_fuse_opts(max_k, mode, precision, tc_min_k, force_path, model, start_qubits, cb, None)
    f = ctypes.c_void_p()
    _check(lib.sv_fuse_circuit(arr, len(gl), n, ctypes.byref(opts), ctypes.byref(f)))
    return f


def sv_fused_free(f) -> None:
    lib.sv_fused_free(f)


def sv_fused_count(f) -> int:
    c = lib.sv_fused_count(f)
    if c < 0:
        _check(c)
    return c


def sv_fused_get_info(f, i: int) -> dict:
    info = sv_fused_info()
    _check(lib.sv_fused_get_info(f, i, ctypes.byref(info)))
    cm = int(info.control_mask)
    return {"k": info.k, "targets": tuple(info.targets[: info.k]), "path": info.path,
            "n_source_gates": info.n_source_gates,
            "controls": tuple(q for q in range(64) if (cm >> q) & 1)}


def sv_fused_get_post_phases(f, i: int) -> list:
    """[(target index, qubit, angle)]: after fused gate i, amplitudes with both bits set get
    exp(i angle)."""
    k = lib.sv_fused_get_post_phases(f, i, 0, None, None, None)
    if k < 0:
        _check(k)
    tg = (ctypes.c_int * max(k, 1))()
    qb = (ctypes.c_int * max(k, 1))()
    an = (ctypes.c_double * max(k, 1))()
    rc = lib.sv_fused_get_post_phases(f, i, k, tg, qb, an)
    if rc < 0:
        _check(rc)
    return [(int(tg[t]), int(qb[t]), float(an[t])) for t in range(k)]


def sv_fused_get_swaps(f, i: int) -> list:
    """[(qubit a, qubit b)]: the disjoint swaps of fused gate i (a swap network), else []."""
    k = lib.sv_fused_get_swaps(f, i, 0, None, None)
    if k < 0:
        _check(k)
    qa = (ctypes.c_int * max(k, 1))()
    qb = (ctypes.c_int * max(k, 1))()
    rc = lib.sv_fused_get_swaps(f, i, k, qa, qb)
    if rc < 0:
        _check(rc)
    return [(int(qa[t]), int(qb[t])) for t in range(k)]


def sv_fused_get_matrix(f, i: int) -> np.ndarray:
    k = sv_fused_get_info(f, i)["k"]
    out = np.zeros((1 << k, 1 << k), dtype=np.complex128)
    _check(lib.sv_fused_get_matrix(f, i, out.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def sv_init_apply(h, basis_index: int, f, timings: bool = False):
    """sv_init followed by sv_apply_fused_gates, started on the small state of the named qubits."""
    if not timings:
        _check(lib.sv_init_apply(h, basis_index, f, None))
        return None
    n = sv_fused_count(f)
    rec = (sv_timing * max(n, 1))()
    _check(lib.sv_init_apply(h, basis_index, f, rec))
    return [{"us": rec[i].us, "k": rec[i].k, "path": rec[i].path, "flags": rec[i].flags,
             "target_mask": rec[i].target_mask} for i in range(n)]


def sv_apply_fused_gates(h, f, timings: bool = False):
    if not timings:
        _check(lib.sv_apply_fused_gates(h, f, None))
        return None
    n = sv_fused_count(f)
    rec = (sv_timing * max(n, 1))()
    _check(lib.sv_apply_fused_gates(h, f, rec))
    return [{"us": rec[i].us, "k": rec[i].k, "path": rec[i].path, "flags": rec[i].flags,
             "target_mask": rec[i].target_mask} for i in range(n)]


# --------------------------------------------------------------------------------------- reductions
def sv_norm(h) -> float:
    out = ctypes.c_double()
    _check(lib.sv_norm(h, ctypes.byref(out)))
    return out.value


def pauli_masks(terms) -> tuple[int, int]:
    """(x_mask, z_mask) of a Pauli string given as {qubit: 'X' | 'Y' | 'Z' | 'I'}."""
    x = z = 0
    for q, s in dict(terms).items():
        s = str(s).upper()
        if s not in ("I", "X", "Y", "Z"):
            raise ValueError(f"unknown Pauli {s!r} on qubit {q}")
        if s in ("X", "Y"):
            x |= 1 << int(q)
        if s in ("Z", "Y"):
            z |= 1 << int(q)
    return x, z


def sv_expval_pauli(h, x_masks, z_masks) -> np.ndarray:
    """<psi|P|psi> for each Pauli string (x_masks[i], z_masks[i]); see pauli_masks."""
    xs = np.ascontiguousarray(np.asarray(x_masks, dtype=np.uint64).reshape(-1))
    zs = np.ascontiguousarray(np.asarray(z_masks, dtype=np.uint64).reshape(-1))
    if xs.size != zs.size:
        raise SvError(SV_EINVAL, "x_masks and z_masks differ in length")
    out = np.zeros(xs.size, dtype=np.float64)
    _check(lib.sv_expval_pauli(h, xs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               zs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), xs.size,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def sv_sample(h, uniforms) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.zeros(u.size, dtype=np.uint64)
    _check(lib.sv_sample(h, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out


def sv_sample_norm(h, uniforms):
    """(samples, norm) from one read pass of the state."""
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.zeros(max(u.size, 1), dtype=np.uint64)
    nrm = ctypes.c_double()
    _check(lib.sv_sample_norm(h, u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(nrm)))
    return out[:u.size], nrm.value


def sv_sample_noalloc(dev_state_ptr: int, n: int, stream: int, uniforms) -> np.ndarray:
    """Sampling through the entry point that allocates no device memory (fixed internal scratch;
    n <= 30, at most 4096 uniforms per call)."""
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.zeros(u.size, dtype=np.uint64)
    _check(lib.sv_sample_noalloc(ctypes.c_void_p(dev_state_ptr), n, ctypes.c_void_p(stream),
                                 u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out


def sv_device_status() -> None:
    _check(lib.sv_device_status())


def sv_version() -> str:
    return lib.sv_version().decode()


# --------------------------------------------------------------------------------------- cost model
def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def sv_mlp_num_params() -> int:
    return int(lib.sv_mlp_num_params())


def sv_mlp_create(seed: int = 1, stream: int = 0):
    h = ctypes.c_void_p()
    _check(lib.sv_mlp_create(ctypes.c_uint64(seed), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def sv_mlp_free(m) -> None:
    lib.sv_mlp_free(m)


def sv_mlp_get_params(m) -> np.ndarray:
    out = np.zeros(sv_mlp_num_params(), dtype=np.float32)
    _check(lib.sv_mlp_get_params(m, _fptr(out)))
    return out


def sv_mlp_set_params(m, params) -> None:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    assert p.size == sv_mlp_num_params()
    _check(lib.sv_mlp_set_params(m, _fptr(p)))


def sv_mlp_features(k: int, targets, path: int, n: int, post_phases: bool = False) -> np.ndarray:
    t = (ctypes.c_int * MAX_K)(*[int(x) for x in targets])
    out = np.zeros(16, dtype=np.float32)
    _check(lib.sv_mlp_features(k, t, path, n, int(bool(post_phases)), _fptr(out)))
    return out


def sv_mlp_gradients(m, X, t):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
    loss = ctypes.c_float()
    g = np.zeros(sv_mlp_num_params(), dtype=np.float32)
    _check(lib.sv_mlp_gradients(m, _fptr(X), _fptr(t), t.size, ctypes.byref(loss), _fptr(g)))
    return loss.value, g


def sv_mlp_adam_step(m, lr: float) -> None:
    _check(lib.sv_mlp_adam_step(m, ctypes.c_float(lr)))


def _stats_dict(st):
    return {f: getattr(st, f) for f, _ in sv_mlp_stats._fields_}


def sv_mlp_train(m, X, us, epochs=200, batch=256, lr=1e-3, seed=1, val_frac=0.1, fallback_k=4) -> dict:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    us = np.ascontiguousarray(np.asarray(us, dtype=np.float32))
    o = sv_mlp_train_opts(epochs, batch, lr, seed, val_frac, fallback_k)
    st = sv_mlp_stats()
    _check(lib.sv_mlp_train(m, _fptr(X), _fptr(us), us.size, ctypes.byref(o), ctypes.byref(st)))
    return _stats_dict(st)


def sv_mlp_predict(m, X) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    out = np.zeros(X.shape[0], dtype=np.float64)
    _check(lib.sv_mlp_predict(m, _fptr(X), X.shape[0], out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def sv_mlp_get_stats(m) -> dict:
    st = sv_mlp_stats()
    _check(lib.sv_mlp_get_stats(m, ctypes.byref(st)))
    return _stats_dict(st)


def sv_mlp_save(m, path: str) -> None:
    _check(lib.sv_mlp_save(m, path.encode()))


def sv_mlp_load(path: str, stream: int = 0):
    h = ctypes.c_void_p()
    _check(lib.sv_mlp_load(path.encode(), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


# --------------------------------------------------------------------------------------- batched circuits
def sv_batch_arena_bytes(ns) -> int:
    a = (ctypes.c_int * len(ns))(*[int(x) for x in ns])
    return int(lib.sv_batch_arena_bytes(a, len(ns)))


def sv_batch_create(fused_list, arena_ptr: int, arena_bytes: int, stream: int = 0):
    arr = (ctypes.c_void_p * len(fused_list))(*[f.value for f in fused_list])
    h = ctypes.c_void_p()
    _check(lib.sv_batch_create(arr, len(fused_list), ctypes.c_void_p(arena_ptr), arena_bytes,
                               ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def sv_batch_free(b) -> None:
    lib.sv_batch_free(b)


def sv_batch_set_opts(b, threads: int, smem_max_n: int, ctas: int, use_graph: bool = True,
                      split_min_n: int = 15, tile_log2: int = 12, wave_mb: int = 0, stage_log2: int = 0,
                      stage_k: int = 0, stage_layers: int = 0, ctas_per_sm: int = 1) -> None:
    o = sv_batch_opts(threads, smem_max_n, ctas, int(bool(use_graph)), split_min_n, tile_log2, wave_mb, stage_log2,
                      stage_k, int(bool(stage_layers)), ctas_per_sm)
    _check(lib.sv_batch_set_opts(b, ctypes.byref(o)))


def sv_batch_get_opts(b) -> dict:
    o = sv_batch_opts()
    _check(lib.sv_batch_get_opts(b, ctypes.byref(o)))
    return {f: getattr(o, f) for f, _ in sv_batch_opts._fields_}


def sv_batch_get_info(b) -> dict:
    o = sv_batch_info()
    _check(lib.sv_batch_get_info(b, ctypes.byref(o)))
    return {f: getattr(o, f) for f, _ in sv_batch_info._fields_}


def sv_batch_run(b) -> None:
    _check(lib.sv_batch_run(b))


def sv_batch_run_loop(b) -> None:
    _check(lib.sv_batch_run_loop(b))


def sv_batch_inject_stall(b, on: bool) -> None:
    _check(lib.sv_batch_inject_stall(b, int(bool(on))))


def sv_batch_plan_stages(f, stage_log2: int) -> list:
    """The stages a batch cuts fused circuit f into (host only): per stage its gate count, local
    qubits, load and store layouts (qubit -> physical bit), and the fused gates it applies."""
    count = sv_fused_count(f)
    k = lib.sv_batch_plan_stages(f, stage_log2, 0, None, None, None, None, None)
    if k < 0:
        _check(k)
    gates = (ctypes.c_int * max(k, 1))()
    lam = (ctypes.c_uint * max(k, 1))()
    lpos = (ctypes.c_int * (32 * max(k, 1)))()
    spos = (ctypes.c_int * (32 * max(k, 1)))()
    order = (ctypes.c_int * max(count, 1))()
    rc = lib.sv_batch_plan_stages(f, stage_log2, k, gates, lam, lpos, spos, order)
    if rc < 0:
        _check(rc)
    out, at = [], 0
    for s in range(k):
        out.append({"gates": list(order[at:at + gates[s]]), "lam": int(lam[s]),
                    "load_pos": list(lpos[32 * s:32 * s + 32]), "store_pos": list(spos[32 * s:32 * s + 32])})
        at += gates[s]
    return out


def sv_batch_state_offset(b, i: int) -> int:
    o = ctypes.c_size_t()
    _check(lib.sv_batch_state_offset(b, i, ctypes.byref(o)))
    return int(o.value)
