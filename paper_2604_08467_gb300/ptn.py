"""Thin ctypes binding of libptn (include/ptn.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; this module
converts circuit descriptions into the C structs, passes torch tensors'
device pointers and the current CUDA stream, and turns status codes into
exceptions.  The library must be built (``build_lib.build()``); importing the
binding without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

from . import build_lib

_HERE = os.path.dirname(os.path.abspath(__file__))

PTN_OK = 0
STATUS_NAMES = {0: "PTN_OK", 1: "PTN_ERR_INVALID_ARG", 2: "PTN_ERR_NOT_CPTP", 3: "PTN_ERR_TOO_LARGE",
                4: "PTN_ERR_OOM", 5: "PTN_ERR_CUDA", 6: "PTN_ERR_TIMEOUT", 7: "PTN_ERR_UNSUPPORTED"}
PTN_PREC_FP32, PTN_PREC_BF16X3, PTN_PREC_FP16X3 = 0, 1, 2
PTN_PROPORTIONAL_FIXED, PTN_PROPORTIONAL_TOTAL, PTN_NONPROP_DIRECT, PTN_NONPROP_EXHAUSTIVE = 0, 1, 2, 3


class PtnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ptn_gate(C.Structure):
    _fields_ = [("arity", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("param_kind", C.c_int32),
                ("param_index", C.c_int32), ("reserved", C.c_int32), ("mat", C.c_double * 32)]


class ptn_circuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_gates", C.c_int32), ("gates", C.POINTER(ptn_gate))]


class ptn_channel(C.Structure):
    _fields_ = [("n_kraus", C.c_int32), ("n_qubits", C.c_int32), ("kraus", C.POINTER(C.c_double))]


class ptn_site(C.Structure):
    _fields_ = [("gate", C.c_int32), ("qubit", C.c_int32), ("channel", C.c_int32)]


class ptn_noise(C.Structure):
    _fields_ = [("n_channels", C.c_int32), ("channels", C.POINTER(ptn_channel)), ("n_sites", C.c_int32),
                ("sites", C.POINTER(ptn_site))]


class ptn_plan_opts(C.Structure):
    _fields_ = [("hypersamples", C.c_int32), ("split_gates", C.c_int32), ("seed", C.c_uint64),
                ("est_traj", C.c_double), ("est_shots", C.c_double), ("mem_cap_bytes", C.c_double),
                ("simt_only", C.c_int32), ("grad_checkpoint", C.c_int32), ("network_form", C.c_int32),
                ("fuse_max", C.c_int32), ("cache_intermediates", C.c_int32), ("keep_products", C.c_int32),
                ("search_threads", C.c_int32)]


class ptn_sample_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("circuit_id", C.c_int32), ("shots_per_traj", C.c_int64),
                ("total_shots", C.c_int64), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("max_traj_per_chunk", C.c_int32), ("use_graphs", C.c_int32), ("reserved", C.c_int32),
                ("branch_shots", C.c_int64), ("final_shots", C.c_int64), ("threshold", C.c_double)]


class ptn_step_stat(C.Structure):
    _fields_ = [("block", C.c_int32), ("step", C.c_int32), ("kernel", C.c_char * 32), ("launches", C.c_int64),
                ("ms", C.c_double), ("alg_bytes", C.c_double), ("alg_flops", C.c_double)]


class ptn_batch_item(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("traj", C.c_void_p), ("opts", ptn_sample_opts)]


class ptn_batch_opts(C.Structure):
    _fields_ = [("n_workers", C.c_int32), ("keep_workspaces", C.c_int32), ("mem_budget_bytes", C.c_double),
                ("max_est_seconds", C.c_double)]


class ptn_pauli_sum(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("coeff", C.POINTER(C.c_double)), ("x_mask", C.POINTER(C.c_uint64)),
                ("z_mask", C.POINTER(C.c_uint64))]


class ptn_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("timed_launches", C.c_int64),
                ("ms", C.c_double), ("alg_bytes", C.c_double), ("alg_flops", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "ptn_plan_path": [C.POINTER(ptn_circuit), C.POINTER(ptn_noise), C.POINTER(C.c_int32), C.c_int32,
                      C.POINTER(ptn_plan_opts), C.POINTER(_P)],
    "ptn_plan_describe": [_P, C.c_int32, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
    "ptn_plan_destroy": [_P],
    "ptn_presample_trajectories": [_P, C.c_uint64, C.c_int32, C.c_int64, C.c_int32, C.POINTER(_P), _P],
    "ptn_presample_range": [_P, C.c_uint64, C.c_int32, C.c_int64, C.c_int64, C.POINTER(_P), _P],
    "ptn_traj_info": [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(_P), C.POINTER(_P),
                      C.POINTER(_P), C.POINTER(_P)],
    "ptn_traj_copy": [_P, _P, _P, _P, _P, _P],
    "ptn_traj_destroy": [_P],
    "ptn_contract_batch": [_P, _P, C.c_int32, _P, _P, C.c_int64, C.c_int32, _P, _P, _P],
    "ptn_sample_block": [_P, C.c_int32, C.c_int32, _P, _P, _P, C.c_int64, C.c_uint64, C.c_int32, C.c_int32,
                         _P, _P, _P, C.c_int64, C.POINTER(C.c_int64), _P],
    "ptn_sample_block_noalloc": [_P, C.c_int32, C.c_int32, _P, _P, _P, C.c_int64, C.c_uint64, C.c_int32,
                                 C.c_int32, _P, _P, _P, C.c_int64, C.POINTER(C.c_int64), _P],
    "ptn_allocate_shots": [_P, C.c_int64, C.c_int64, C.c_uint64, C.c_int32, _P, _P],
    "ptn_sample_shots": [_P, _P, C.POINTER(ptn_sample_opts), C.POINTER(_P), _P],
    "ptn_shots_info": [_P, C.POINTER(C.c_int64), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                       C.POINTER(C.c_int64), C.c_int32],
    "ptn_shots_copy": [_P, _P, _P, _P, _P],
    "ptn_shots_destroy": [_P],
    "ptn_shots_probs": [_P, C.POINTER(_P)],
    "ptn_shots_copy_probs": [_P, _P, _P],
    "ptn_shots_merge": [_P, C.POINTER(_P), _P],
    "ptn_sample_shots_batch": [C.POINTER(ptn_batch_item), C.c_int32, C.POINTER(ptn_batch_opts), C.POINTER(_P),
                               C.POINTER(C.c_int), _P],
    "ptn_expval_grad": [_P, _P, C.POINTER(ptn_pauli_sum), C.POINTER(C.c_double), C.c_int32, _P, _P, _P],
    "ptn_trajectory_amplitudes": [_P, _P, C.c_int64, C.c_int64, C.c_int32, _P, _P],
    "ptn_set_wait_limit": [C.c_double],
    "ptn_tune_tiles": [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                       C.c_void_p],
    "ptn_tune_block_sizes": [C.POINTER(ptn_circuit), C.POINTER(ptn_noise), C.POINTER(C.c_int32), C.c_int32,
                             C.POINTER(ptn_plan_opts), C.c_int64, C.c_int64, C.c_uint64, C.POINTER(C.c_int32),
                             C.POINTER(C.c_double), _P],
    "ptn_stats_enable": [C.c_int32],
    "ptn_stats_enable_only": [C.c_char_p],
    "ptn_stats_reset": [],
    "ptn_stats_read": [C.POINTER(ptn_kernel_stat), C.c_int32, C.POINTER(C.c_int32)],
    "ptn_stats_read_steps": [C.POINTER(ptn_step_stat), C.c_int32, C.POINTER(C.c_int32)],
    "ptn_status_string": [C.c_int],
    "ptn_last_error": [],
    "ptn_version": [],
}
_RESTYPE = {"ptn_plan_destroy": None, "ptn_traj_destroy": None, "ptn_shots_destroy": None,
            "ptn_status_string": C.c_char_p, "ptn_last_error": C.c_char_p, "ptn_version": C.c_char_p}

_lib_handle = None
last_batch_error = ""


def library_path():
    return build_lib.LIB


def lib():
    """Load libptn.so (building it first if sources are newer)."""
    global _lib_handle
    if _lib_handle is None:
        path = build_lib.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libptn.so not found at {path}")
        h = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(h, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, C.c_int)
        _lib_handle = h
    return _lib_handle


def exported_symbols():
    return sorted(_SIGS)


def _check(status):
    if status != PTN_OK:
        raise PtnError(status, lib().ptn_last_error().decode())


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else int(t.data_ptr()))


# ------------------------------------------------------------ marshalling --

def circuit_structs(circ):
    """workloads.Circuit -> (ptn_circuit, ptn_noise, keepalive)."""
    n_g = len(circ.gates)
    gates = (ptn_gate * max(n_g, 1))()
    for l, g in enumerate(circ.gates):
        gs = gates[l]
        gs.arity = g.arity
        gs.q0 = g.qubits[0]
        gs.q1 = g.qubits[1] if g.arity == 2 else -1
        gs.param_kind = int(getattr(g, "param_kind", 0))
        gs.param_index = int(getattr(g, "param_index", -1))
        m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
        flat = np.empty(2 * m.size)
        flat[0::2], flat[1::2] = m.real, m.imag
        for k, v in enumerate(flat):
            gs.mat[k] = float(v)
    c = ptn_circuit(circ.n_qubits, n_g, gates)
    n_ch = len(circ.channels)
    chans = (ptn_channel * max(n_ch, 1))()
    kraus_arrays = []
    for k, ch in enumerate(circ.channels):
        arr = np.concatenate([np.stack([np.asarray(K, np.complex128).reshape(-1).real,
                                        np.asarray(K, np.complex128).reshape(-1).imag], axis=1).reshape(-1)
                              for K in ch.kraus]).astype(np.float64)
        kraus_arrays.append(arr)
        chans[k].n_kraus = len(ch.kraus)
        chans[k].n_qubits = 2 if np.asarray(ch.kraus[0]).shape[0] == 4 else 1
        chans[k].kraus = arr.ctypes.data_as(C.POINTER(C.c_double))
    n_s = len(circ.sites)
    sites = (ptn_site * max(n_s, 1))()
    for s, st in enumerate(circ.sites):
        sites[s].gate, sites[s].qubit, sites[s].channel = st.gate, st.qubit, st.channel
    nz = ptn_noise(n_ch, chans, n_s, sites)
    return c, nz, (gates, chans, kraus_arrays, sites)


# -------------------------------------------------------------- handles ----

class Plan:
    def __init__(self, handle, n_qubits, block_sizes):
        self.handle = handle
        self.n_qubits = n_qubits
        self.block_sizes = list(block_sizes)
        s, self.blocks = 0, []
        for b in self.block_sizes:
            self.blocks.append((s, b))
            s += b

    def describe(self, detail=0):
        n = C.c_size_t(0)
        _check(lib().ptn_plan_describe(self.handle, detail, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        _check(lib().ptn_plan_describe(self.handle, detail, buf, n.value + 1, C.byref(n)))
        return json.loads(buf.value.decode())

    def __del__(self):
        if getattr(self, "handle", None) and _lib_handle is not None:
            _lib_handle.ptn_plan_destroy(self.handle)
            self.handle = None


class Traj:
    def __init__(self, handle, plan):
        self.handle = handle
        self.plan = plan
        n = C.c_int64(0)
        S = C.c_int32(0)
        _check(lib().ptn_traj_info(handle, C.byref(n), C.byref(S), None, None, None, None))
        self.n_unique = n.value
        self.n_sites = S.value

    def to_torch(self, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        kr = torch.empty((self.n_unique, self.n_sites), dtype=torch.uint8, device=dev)
        lq = torch.empty(self.n_unique, dtype=torch.float64, device=dev)
        mu = torch.empty(self.n_unique, dtype=torch.int64, device=dev)
        fi = torch.empty(self.n_unique, dtype=torch.int64, device=dev)
        _check(lib().ptn_traj_copy(self.handle, _ptr(kr), _ptr(lq), _ptr(mu), _ptr(fi), _stream(stream)))
        return kr, lq, mu, fi

    def __del__(self):
        if getattr(self, "handle", None) and _lib_handle is not None:
            _lib_handle.ptn_traj_destroy(self.handle)
            self.handle = None


def words_of(n_qubits):
    """64-bit words per bitstring of an n-qubit plan."""
    return (int(n_qubits) + 63) // 64


def bits_to_int(words):
    """The Python integer of one bitstring given as its little-endian words."""
    w = [int(x) & 0xFFFFFFFFFFFFFFFF for x in (words if hasattr(words, "__len__") else [words])]
    return sum(x << (64 * i) for i, x in enumerate(w))


def int_to_words(values, n_words):
    """int64 array [len(values), n_words] of the little-endian words of each
    Python integer (for prefixes of wide plans)."""
    import numpy as np
    out = np.zeros((len(values), n_words), dtype=np.uint64)
    for i, v in enumerate(values):
        v = int(v)
        for w in range(n_words):
            out[i, w] = (v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF
    return out.view(np.int64)


class Shots:
    """A sampling result.  Bitstrings are n_words = ceil(n_qubits / 64)
    little-endian uint64 words each (held as int64); to_torch gives them as
    [n] for one word and [n, n_words] otherwise."""

    def __init__(self, handle, n_blocks, n_words=1):
        self.handle = handle
        self.n_words = int(n_words)
        n = C.c_int64(0)
        nets = (C.c_int64 * max(n_blocks, 1))()
        _check(lib().ptn_shots_info(handle, C.byref(n), None, None, None, nets, n_blocks))
        self.n = n.value
        self.nets_per_block = [nets[j] for j in range(n_blocks)]

    def to_torch(self, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        t = torch.empty(self.n, dtype=torch.int32, device=dev)
        b = torch.empty((self.n, self.n_words) if self.n_words > 1 else (self.n,), dtype=torch.int64, device=dev)
        c = torch.empty(self.n, dtype=torch.int64, device=dev)
        _check(lib().ptn_shots_copy(self.handle, _ptr(t), _ptr(b), _ptr(c), _stream(stream)))
        return t, b, c

    def probs(self, stream=None):
        """Per-record probabilities p(x | prefix) (non-proportional results)."""
        import torch
        p = torch.empty(self.n, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
        _check(lib().ptn_shots_copy_probs(self.handle, _ptr(p), _stream(stream)))
        return p

    def __del__(self):
        if getattr(self, "handle", None) and _lib_handle is not None:
            _lib_handle.ptn_shots_destroy(self.handle)
            self.handle = None


# ------------------------------------------------------------------ calls ----

def ptn_plan_path(circ, block_sizes=None, hypersamples=100, split_gates=1, seed=1234, est_traj=1024,
                  est_shots=1e6, mem_cap_bytes=0.0, simt_only=False, grad_checkpoint=False, network_form=0,
                  fuse_max=0, cache_intermediates=True, keep_products=False, search_threads=0):
    """Plan a circuit (ptn_plan_opts in include/ptn.h).  Intermediate caching
    across error sets is on by default here (results are bit-identical with
    it off; the C structure's zero value is off)."""
    c, nz, keep = circuit_structs(circ)
    if block_sizes is None:
        n = circ.n_qubits
        f = -(-n // 10)
        block_sizes = [10] * (f - 1) + [n - 10 * (f - 1)]
    bs = (C.c_int32 * len(block_sizes))(*block_sizes)
    opts = ptn_plan_opts(hypersamples, split_gates, seed, float(est_traj), float(est_shots), float(mem_cap_bytes),
                         int(bool(simt_only)), int(bool(grad_checkpoint)), int(network_form), int(fuse_max),
                         int(bool(cache_intermediates)), int(bool(keep_products)), int(search_threads))
    h = C.c_void_p()
    _check(lib().ptn_plan_path(C.byref(c), C.byref(nz), bs, len(block_sizes), C.byref(opts), C.byref(h)))
    del keep
    return Plan(h, circ.n_qubits, block_sizes)


def ptn_presample_trajectories(plan, seed, n_traj, dedup=False, circuit_id=0, stream=None):
    h = C.c_void_p()
    _check(lib().ptn_presample_trajectories(plan.handle, seed, circuit_id, n_traj, int(bool(dedup)),
                                            C.byref(h), _stream(stream)))
    return Traj(h, plan)


def ptn_presample_range(plan, seed, traj0, n_traj, circuit_id=0, stream=None):
    """Trajectories traj0 .. traj0 + n_traj - 1 of the draw made from `seed`
    (global Philox counters, no dedup)."""
    h = C.c_void_p()
    _check(lib().ptn_presample_range(plan.handle, seed, circuit_id, int(traj0), int(n_traj), C.byref(h),
                                     _stream(stream)))
    return Traj(h, plan)


def ptn_contract_batch(plan, traj, block, net_traj, net_prefix, marg_out, Z_out, precision=PTN_PREC_FP32,
                       stream=None):
    n = int(net_traj.numel())
    w = words_of(plan.n_qubits)
    if int(net_prefix.numel()) < n * w:
        raise ValueError(f"net_prefix needs {w} words per network ({n * w} entries)")
    if int(marg_out.numel()) < n << plan.block_sizes[block] or int(Z_out.numel()) < n:
        raise ValueError("marg_out / Z_out shorter than n_net networks need")
    _check(lib().ptn_contract_batch(plan.handle, traj.handle, block, _ptr(net_traj), _ptr(net_prefix), n,
                                    precision, _ptr(marg_out), _ptr(Z_out), _stream(stream)))


def _sample_block_sizes(marg, b, parent_traj, parent_prefix, parent_count, child_traj, child_prefix, child_count):
    """(n_parent, child_cap) of a sampling call, checked against every buffer
    the library reads or writes (device buffers are not bounds-checked)."""
    n = int(parent_traj.numel())
    if int(parent_prefix.numel()) < n or int(parent_count.numel()) < n:
        raise ValueError("parent_prefix / parent_count shorter than parent_traj")
    if int(marg.numel()) != n << b:
        raise ValueError(f"marg has {int(marg.numel())} entries, expected n_parent * 2^b = {n << b}")
    cap = min(int(child_traj.numel()), int(child_prefix.numel()), int(child_count.numel()))
    return n, cap


def ptn_sample_block(marg, b, start, parent_traj, parent_prefix, parent_count, seed, circuit_id, block,
                     child_traj, child_prefix, child_count, stream=None):
    n, cap = _sample_block_sizes(marg, b, parent_traj, parent_prefix, parent_count, child_traj, child_prefix,
                                 child_count)
    nc = C.c_int64(0)
    _check(lib().ptn_sample_block(_ptr(marg), b, start, _ptr(parent_traj), _ptr(parent_prefix),
                                  _ptr(parent_count), n, seed, circuit_id, block,
                                  _ptr(child_traj), _ptr(child_prefix), _ptr(child_count),
                                  cap, C.byref(nc), _stream(stream)))
    return nc.value


def ptn_sample_block_noalloc(marg, b, start, parent_traj, parent_prefix, parent_count, seed, circuit_id, block,
                             child_traj, child_prefix, child_count, stream=None):
    """ptn_sample_block with its scratch in the library's fixed static device
    array (no allocation during the call; see include/ptn.h)."""
    n, cap = _sample_block_sizes(marg, b, parent_traj, parent_prefix, parent_count, child_traj, child_prefix,
                                 child_count)
    nc = C.c_int64(0)
    _check(lib().ptn_sample_block_noalloc(_ptr(marg), b, start, _ptr(parent_traj), _ptr(parent_prefix),
                                          _ptr(parent_count), n, seed, circuit_id, block,
                                          _ptr(child_traj), _ptr(child_prefix), _ptr(child_count),
                                          cap, C.byref(nc), _stream(stream)))
    return nc.value


def ptn_allocate_shots(weights, total, seed, circuit_id, m_out, stream=None):
    _check(lib().ptn_allocate_shots(_ptr(weights), int(weights.numel()), int(total), seed, circuit_id,
                                    _ptr(m_out), _stream(stream)))


def ptn_sample_shots(plan, traj, seed, shots_per_traj=None, total_shots=None, circuit_id=0,
                     precision=PTN_PREC_FP32, max_traj_per_chunk=0, use_graphs=0, stream=None):
    o = _sample_opts(seed, shots_per_traj, total_shots, circuit_id, precision, max_traj_per_chunk)
    o.use_graphs = use_graphs
    h = C.c_void_p()
    _check(lib().ptn_sample_shots(plan.handle, traj.handle, C.byref(o), C.byref(h), _stream(stream)))
    return Shots(h, len(plan.block_sizes), words_of(plan.n_qubits))


def _sample_opts(seed, shots_per_traj=None, total_shots=None, circuit_id=0, precision=PTN_PREC_FP32,
                 max_traj_per_chunk=0):
    mode = PTN_PROPORTIONAL_FIXED if total_shots is None else PTN_PROPORTIONAL_TOTAL
    return ptn_sample_opts(mode, circuit_id, int(shots_per_traj or 0), int(total_shots or 0), seed, precision,
                           max_traj_per_chunk, 0, 0, 0, 0, 0.0)


def ptn_sample_nonprop(plan, traj, seed, mode="exhaustive", branch_shots=1, final_shots=0, threshold=0.0,
                       circuit_id=0, precision=PTN_PREC_FP32, max_traj_per_chunk=0, use_graphs=0, stream=None):
    """Non-proportional NBS (include/ptn.h): branch_shots per prefix on the
    non-final blocks, then the final block harvested directly (final_shots
    draws per network) or exhaustively (p(x | prefix) >= threshold)."""
    code = {"direct": PTN_NONPROP_DIRECT, "exhaustive": PTN_NONPROP_EXHAUSTIVE}[mode]
    o = ptn_sample_opts(code, circuit_id, 0, 0, seed, precision, max_traj_per_chunk, int(use_graphs), 0, int(branch_shots),
                        int(final_shots), float(threshold))
    h = C.c_void_p()
    _check(lib().ptn_sample_shots(plan.handle, traj.handle, C.byref(o), C.byref(h), _stream(stream)))
    return Shots(h, len(plan.block_sizes), words_of(plan.n_qubits))


def ptn_sample_shots_batch(items, n_workers=4, keep_workspaces=False, mem_budget_bytes=0.0, max_est_seconds=0.0,
                           stream=None):
    """Mixed-circuit batch (include/ptn.h).  items: list of dicts with keys
    plan, traj, seed and shots_per_traj or total_shots (optional circuit_id,
    precision).  Returns a list of (status, Shots or None) in item order."""
    n = len(items)
    arr = (ptn_batch_item * max(n, 1))()
    for i, it in enumerate(items):
        arr[i].plan = it["plan"].handle
        arr[i].traj = it["traj"].handle
        arr[i].opts = _sample_opts(it["seed"], it.get("shots_per_traj"), it.get("total_shots"),
                                   it.get("circuit_id", 0), it.get("precision", PTN_PREC_FP32))
    bo = ptn_batch_opts(n_workers, int(bool(keep_workspaces)), float(mem_budget_bytes), float(max_est_seconds))
    outs = (C.c_void_p * max(n, 1))()
    sts = (C.c_int * max(n, 1))()
    _check(lib().ptn_sample_shots_batch(arr, n, C.byref(bo), outs, sts, _stream(stream)))
    global last_batch_error
    last_batch_error = lib().ptn_last_error().decode()   # first failing item's message, if any
    res = []
    for i, it in enumerate(items):
        if sts[i] == PTN_OK:
            res.append((PTN_OK, Shots(C.c_void_p(outs[i]), len(it["plan"].block_sizes),
                                      words_of(it["plan"].n_qubits))))
        else:
            res.append((sts[i], None))
    return res


def ptn_expval_grad(plan, traj, terms, theta, value_out, grad_out, stream=None):
    """Trajectory-averaged <O> and dO/dtheta (include/ptn.h).  terms: list of
    (coeff, z_mask) or (coeff, x_mask, z_mask); theta: host sequence of angles;
    value_out: device float64 [1]; grad_out: device float64 [len(theta)]."""
    n_t = len(terms)
    coeff = (C.c_double * max(n_t, 1))()
    xm = (C.c_uint64 * max(n_t, 1))()
    zm = (C.c_uint64 * max(n_t, 1))()
    for t, term in enumerate(terms):
        coeff[t] = float(term[0])
        xm[t] = int(term[1]) if len(term) == 3 else 0
        zm[t] = int(term[-1])
    obs = ptn_pauli_sum(n_t, coeff, xm, zm)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    thp = th.ctypes.data_as(C.POINTER(C.c_double)) if th.size else None
    _check(lib().ptn_expval_grad(plan.handle, traj.handle, C.byref(obs), thp, int(th.size), _ptr(value_out),
                                 _ptr(grad_out), _stream(stream)))


def ptn_trajectory_amplitudes(plan, traj, traj0, n_traj, amp_out, precision=PTN_PREC_FP32, stream=None):
    """<x|psi_i> for distinct error sets traj0 .. traj0 + n_traj - 1 into the
    device complex64 tensor amp_out of shape [n_traj, 2^n] (include/ptn.h)."""
    if int(amp_out.numel()) != n_traj << plan.n_qubits or amp_out.element_size() != 8:
        raise ValueError("amp_out must be complex64 with n_traj * 2^n entries")
    _check(lib().ptn_trajectory_amplitudes(plan.handle, traj.handle, int(traj0), int(n_traj), precision,
                                           _ptr(amp_out), _stream(stream)))


def ptn_shots_merge(shots, n_blocks, stream=None):
    """Shots merged across trajectories (include/ptn.h): one record per distinct
    bitstring, increasing bits, traj = -1."""
    h = C.c_void_p()
    _check(lib().ptn_shots_merge(shots.handle, C.byref(h), _stream(stream)))
    return Shots(h, n_blocks, shots.n_words)


def ptn_tune_block_sizes(circ, candidates, probe_traj, probe_shots, seed=1, hypersamples=16, split_gates=1,
                         plan_seed=1234, stream=None):
    """Fastest block size among `candidates` by timed probe runs (include/ptn.h).
    Returns (best b, [seconds per candidate])."""
    c, nz, keep = circuit_structs(circ)
    opts = ptn_plan_opts(hypersamples, split_gates, plan_seed, float(probe_traj), float(probe_shots), 0.0, 0, 0, 0,
                         0)
    cand = (C.c_int32 * len(candidates))(*candidates)
    secs = (C.c_double * len(candidates))()
    best = C.c_int32(0)
    _check(lib().ptn_tune_block_sizes(C.byref(c), C.byref(nz), cand, len(candidates), C.byref(opts), int(probe_traj),
                                      int(probe_shots), seed, C.byref(best), secs, _stream(stream)))
    del keep
    return best.value, [secs[i] for i in range(len(candidates))]


def ptn_tune_tiles(plan, traj, n_probe=64, reps=3, stream=None):
    """Time every SIMT step of the plan under each micro-tile shape on a probe
    of n_probe networks and keep the fastest (include/ptn.h).  Returns
    (steps timed, steps whose shape changed from the default)."""
    nt, nc = C.c_int32(0), C.c_int32(0)
    _check(lib().ptn_tune_tiles(plan.handle, traj.handle, int(n_probe), int(reps), C.byref(nt), C.byref(nc),
                                _stream(stream)))
    return nt.value, nc.value


def ptn_set_wait_limit(seconds):
    """Limit of the tensor-core kernel's pipeline waits (default 2 s)."""
    _check(lib().ptn_set_wait_limit(float(seconds)))


def ptn_stats_enable(on=True):
    _check(lib().ptn_stats_enable(int(bool(on))))


def ptn_stats_enable_only(kernel):
    """Time only the launches of one kernel class (others are just counted)."""
    _check(lib().ptn_stats_enable_only(kernel.encode() if kernel else None))


def ptn_stats_reset():
    _check(lib().ptn_stats_reset())


def ptn_stats_read():
    """{kernel name: dict(launches, timed_launches, ms, alg_bytes, alg_flops)} (synchronises)."""
    buf = (ptn_kernel_stat * 32)()
    n = C.c_int32(0)
    _check(lib().ptn_stats_read(buf, 32, C.byref(n)))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, timed_launches=buf[i].timed_launches,
                                       ms=buf[i].ms, alg_bytes=buf[i].alg_bytes, alg_flops=buf[i].alg_flops)
            for i in range(n.value)}


def ptn_stats_read_steps():
    """[(block, step, kernel, launches, ms, alg_bytes, alg_flops)] (synchronises)."""
    n = C.c_int32(0)
    _check(lib().ptn_stats_read_steps(None, 1 << 30, C.byref(n)))
    buf = (ptn_step_stat * max(n.value, 1))()
    _check(lib().ptn_stats_read_steps(buf, n.value, C.byref(n)))
    return [(r.block, r.step, r.kernel.decode(), r.launches, r.ms, r.alg_bytes, r.alg_flops)
            for r in buf[:n.value]]
