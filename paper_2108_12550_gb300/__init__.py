"""Python binding of librmdec: GPU p-FHT-FSCL-L-M decoding of Reed-Muller codes
(arXiv 2108.12550) and the Aut-SSC-P baseline.

This module only marshals arguments to the C ABI declared in ``include/rmdec.h``; every
decoding step runs in the library's CUDA kernels. PyTorch supplies device memory and
streams. Importing fails loudly if the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librmdec.so")

OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEDOUT, EDEVICE, ECANCELED = 0, -1, -2, -3, -4, -5, -6, -7
DTYPES = {"f32": 0, "i8": 1, "f16": 2, "i16": 3}
PERM_REC = 11

_lib = None


class _Segment(ctypes.Structure):
    """rmdec_segment (include/rmdec_group.h)."""
    _fields_ = [("decoder", ctypes.c_int), ("llr_dev", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("bits_out_dev", ctypes.c_void_p)]


class RmdecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rmdec status {status}: {msg}")
        self.status = status


def load_library():
    """Loads librmdec.so (built by ``paper_2108_12550_gb300._build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    V, I, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "rmdec_create": ([ctypes.POINTER(V), I, I, I, I, U64], I),
        "rmdec_create_aut_ssc": ([ctypes.POINTER(V), I, I, I, U64], I),
        "rmdec_create_fhtfscl": ([ctypes.POINTER(V), I, I, I], I),
        "rmdec_destroy": ([V], None),
        "rmdec_set_dtype": ([V, I], I),
        "rmdec_set_hadamard": ([V, I], I),
        "rmdec_set_kernel": ([V, I], I),
        "rmdec_kernel_for": ([V, I64, ctypes.POINTER(I)], I),
        "rmdec_perm_count": ([V, ctypes.POINTER(I64)], I),
        "rmdec_get_perms": ([V, V, I64], I),
        "rmdec_set_perms": ([V, V, I64], I),
        "rmdec_info": ([V, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.POINTER(I))], I),
        "rmdec_decode": ([V, V, I64, V, V], I),
        "rmdec_decode_debug": ([V, V, I64, V, V, V, V, V], I),
        "rmdec_decode_host": ([V, V, I64, V, V], I),
        "rmdec_decode_noalloc": ([V, V, I64, V, V], I),
        "rmdec_submit": ([V, V, I64, V, V, ctypes.POINTER(U64)], I),
        "rmdec_poll": ([V, U64, I64], I),
        "rmdec_last_error": ([V], ctypes.c_char_p),
        "rmdec_set_tuning": ([V, I, I], I),
        "rmdec_get_tuning": ([V, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "rmdec_autotune": ([V, I64, ctypes.c_char_p, V], I),
        "rmdec_graph_create": ([V, V, I64, V, ctypes.POINTER(V)], I),
        "rmdec_graph_launch": ([V, V], I),
        "rmdec_graph_destroy": ([V], None),
        "rmdec_debug_fail_device_allocs": ([I64], I),
        "rmdec_group_create": ([ctypes.POINTER(V), ctypes.POINTER(V), I], I),
        "rmdec_group_decode": ([V, ctypes.POINTER(_Segment), I, V], I),
        "rmdec_group_set_tuning": ([V, I, I], I),
        "rmdec_group_set_split": ([V, I64], I),
        "rmdec_group_destroy": ([V], None),
        "rmdec_group_last_error": ([V], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


class Decoder:
    """A decoder handle. algo='pfht' (p-FHT-FSCL-L-P, Algorithm 5), 'fhtfscl' (FHT-FSCL-L, no
    permutations; P must be 1) or 'autssc' (Aut-SSC-P)."""

    def __init__(self, m, r, P, L=1, perm_seed=0, dtype="f32", perms=None, algo="pfht"):
        lib = load_library()
        self._lib = lib
        h = ctypes.c_void_p()
        if algo == "pfht":
            st = lib.rmdec_create(ctypes.byref(h), m, r, P, L, perm_seed)
        elif algo == "autssc":
            st = lib.rmdec_create_aut_ssc(ctypes.byref(h), m, r, P, perm_seed)
        elif algo == "fhtfscl":
            st = lib.rmdec_create_fhtfscl(ctypes.byref(h), m, r, L)
        else:
            raise ValueError(algo)
        if st != OK:
            raise RmdecError(st, lib.rmdec_last_error(None).decode())
        self._h = h
        self.m, self.r, self.P, self.L, self.algo = m, r, P, (1 if algo == "autssc" else L), algo
        n, k = ctypes.c_int(), ctypes.c_int()
        idx = ctypes.POINTER(ctypes.c_int)()
        self._check(lib.rmdec_info(h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(idx)))
        self.n, self.k = n.value, k.value
        self.info_idx = np.array([idx[i] for i in range(self.k)], dtype=np.int64)
        self.kw = (self.k + 31) // 32
        self.nw = max(1, self.n // 32)
        self.dtype = None
        self.set_dtype(dtype)
        if perms is not None:
            self.set_perms(perms)

    def _check(self, st):
        if st != OK:
            raise RmdecError(st, self._lib.rmdec_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rmdec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_dtype(self, dtype):
        self._check(self._lib.rmdec_set_dtype(self._h, DTYPES[dtype]))
        self.dtype = dtype

    def set_hadamard(self, mode):
        """'shuffle' (FP32 butterflies, default) or 'tensor' (FP16 tensor-core products)."""
        self._check(self._lib.rmdec_set_hadamard(self._h, {"shuffle": 0, "tensor": 1}[mode]))
        self.hadamard = mode

    def set_kernel(self, kernel):
        """'auto' (default: 'warp', and 'path' for large launches where it exists), 'warp' (one
        warp per decoder) or 'path' (one thread per list path, RM(2, m) with 4 <= m <= 8 or
        RM(3, m) with 5 <= m <= 7, and L <= 8)."""
        self._check(self._lib.rmdec_set_kernel(self._h, {"auto": 0, "warp": 1, "path": 2}[kernel]))
        self.kernel = kernel

    def kernel_for(self, n_frames):
        """'path' or 'warp': the kernel that decodes a launch of n_frames frames now."""
        k = ctypes.c_int()
        self._check(self._lib.rmdec_kernel_for(self._h, ctypes.c_int64(n_frames), ctypes.byref(k)))
        return {1: "warp", 2: "path"}[k.value]

    def perm_count(self):
        n = ctypes.c_int64()
        self._check(self._lib.rmdec_perm_count(self._h, ctypes.byref(n)))
        return n.value

    def get_perms(self):
        n = self.perm_count()
        out = np.zeros((n, PERM_REC), dtype=np.uint16)
        self._check(self._lib.rmdec_get_perms(self._h, out.ctypes.data, n))
        return out

    def set_perms(self, perms):
        a = np.ascontiguousarray(perms, dtype=np.uint16).reshape(-1, PERM_REC)
        self._check(self._lib.rmdec_set_perms(self._h, a.ctypes.data, a.shape[0]))

    def _alloc_bits(self, F, out):
        import torch
        if out is None:
            out = torch.empty((F, self.kw), dtype=torch.int32, device="cuda")
        return out

    def decode(self, llr, out=None, stream=None):
        """llr: CUDA tensor [F, n] of the handle's dtype. Returns int32 [F, ceil(k/32)]."""
        F = llr.shape[0]
        out = self._alloc_bits(F, out)
        self._check(self._lib.rmdec_decode(self._h, _ptr(llr), F, _ptr(out), _stream_ptr(stream)))
        return out

    def decode_noalloc(self, llr, out, stream=None):
        """rmdec_decode_noalloc: as decode, but the library allocates no device memory (its
        tables go to a fixed device array shared by all such calls; see include/rmdec.h).
        The caller supplies `out` (int32 CUDA tensor [F, ceil(k/32)])."""
        self._check(self._lib.rmdec_decode_noalloc(self._h, _ptr(llr), llr.shape[0], _ptr(out),
                                                   _stream_ptr(stream)))
        return out

    def decode_debug(self, llr, stream=None):
        import torch
        F = llr.shape[0]
        bits = self._alloc_bits(F, None)
        cw = torch.empty((F, self.nw), dtype=torch.int32, device="cuda")
        pm = torch.empty(F, dtype=torch.float32, device="cuda")
        best = torch.empty(F, dtype=torch.int32, device="cuda")
        self._check(self._lib.rmdec_decode_debug(self._h, _ptr(llr), F, _ptr(bits), _ptr(cw), _ptr(pm),
                                                 _ptr(best), _stream_ptr(stream)))
        return bits, cw, pm, best

    def decode_host(self, llr_host, out_host, stream=None):
        """Host-to-host decode (copies inside): llr_host/out_host are CPU tensors (pinned for speed)."""
        self._check(self._lib.rmdec_decode_host(self._h, llr_host.data_ptr(), llr_host.shape[0],
                                                out_host.data_ptr(), _stream_ptr(stream)))
        return out_host

    def set_tuning(self, warps_per_cta=0, ctas_per_sm=0):
        self._check(self._lib.rmdec_set_tuning(self._h, warps_per_cta, ctas_per_sm))

    def get_tuning(self):
        w, c = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.rmdec_get_tuning(self._h, ctypes.byref(w), ctypes.byref(c)))
        return w.value, c.value

    def autotune(self, n_frames=16384, cache_path=None, stream=None):
        cp = cache_path.encode() if cache_path else None
        self._check(self._lib.rmdec_autotune(self._h, n_frames, cp, _stream_ptr(stream)))
        return self.get_tuning()

    def graph(self, llr_host, out_host):
        """A captured host-to-host decode (H2D, decode, D2H) for these fixed CPU buffers."""
        return Graph(self, llr_host, out_host)

    def submit(self, llr, out, stream=None):
        t = ctypes.c_uint64()
        self._check(self._lib.rmdec_submit(self._h, _ptr(llr), llr.shape[0], _ptr(out), _stream_ptr(stream),
                                           ctypes.byref(t)))
        return t.value

    def poll(self, ticket, timeout_us=0):
        """Returns OK, EBUSY or ETIMEDOUT (other statuses raise)."""
        st = self._lib.rmdec_poll(self._h, ticket, int(timeout_us))
        if st in (OK, EBUSY, ETIMEDOUT):
            return st
        return self._check(st)


class Graph:
    """rmdec_graph_t: one replay = H2D of the LLRs, decode, D2H of the bits."""

    def __init__(self, dec, llr_host, out_host):
        self._dec = dec
        self._lib = dec._lib
        self._bufs = (llr_host, out_host)  # the host buffers must outlive the graph
        g = ctypes.c_void_p()
        dec._check(self._lib.rmdec_graph_create(dec._h, llr_host.data_ptr(), llr_host.shape[0],
                                                out_host.data_ptr(), ctypes.byref(g)))
        self._g = g

    def launch(self, stream=None):
        self._dec._check(self._lib.rmdec_graph_launch(self._g, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_g", None):
            self._lib.rmdec_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """rmdec_group_t: one kernel launch over frames of several decoders (include/rmdec_group.h).
    The decoders must be p-FHT-FSCL or FHT-FSCL handles with one list size L in {1, 2, 4, 8}."""

    def __init__(self, decoders):
        lib = load_library()
        self._lib = lib
        arr = (ctypes.c_void_p * len(decoders))(*[d._h.value for d in decoders])
        h = ctypes.c_void_p()
        st = lib.rmdec_group_create(ctypes.byref(h), arr, len(decoders))
        if st != OK:
            raise RmdecError(st, lib.rmdec_group_last_error(None).decode())
        self._h = h
        self._decoders = list(decoders)  # the handles must outlive the group

    def _check(self, st):
        if st != OK:
            raise RmdecError(st, self._lib.rmdec_group_last_error(self._h).decode())
        return st

    def decode(self, segments, stream=None):
        """segments: list of (decoder index, llr CUDA tensor [F, n] of that decoder's dtype,
        out CUDA int32 tensor [F, ceil(k/32)] or None). Returns the output tensors."""
        arr = (_Segment * max(1, len(segments)))()
        outs = []
        for i, (d, llr, out) in enumerate(segments):
            if out is None:
                out = self._decoders[d]._alloc_bits(llr.shape[0], None)
            arr[i] = _Segment(d, _ptr(llr), llr.shape[0], _ptr(out))
            outs.append(out)
        self._check(self._lib.rmdec_group_decode(self._h, arr, len(segments), _stream_ptr(stream)))
        return outs

    def set_tuning(self, warps_per_cta=0, ctas_per_sm=0):
        """Launch shape of the grouped launches: warps per CTA (1..20; 0 = the default, with
        wide CTAs for launches of at most one wave) and a cap on CTAs per SM (0 = occupancy).
        Never changes results."""
        self._check(self._lib.rmdec_group_set_tuning(self._h, warps_per_cta, ctas_per_sm))

    def set_split(self, min_frames_alone=0):
        """Segments of at least this many frames run in their own decoder's launch (0: one full
        wave of that launch; negative: every segment stays in the grouped launch)."""
        self._check(self._lib.rmdec_group_set_split(self._h, int(min_frames_alone)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rmdec_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_fail_device_allocs(n):
    """Test hook: the library's next n device allocations fail as if out of memory (0 disarms)."""
    st = load_library().rmdec_debug_fail_device_allocs(int(n))
    if st != OK:
        raise RmdecError(st, "bad count")


def unpack_bits(words, nbits):
    """[F, W] int32/uint32 words -> [F, nbits] uint8 (bit j = bit j%32 of word j//32)."""
    w = np.asarray(words).astype(np.uint32)
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(w.shape[0], -1)[:, :nbits].astype(np.uint8)


def pack_bits(bits):
    """[F, nbits] 0/1 -> [F, ceil(nbits/32)] uint32."""
    b = np.asarray(bits, dtype=np.uint32)
    F, n = b.shape
    W = (n + 31) // 32
    pad = np.zeros((F, W * 32), dtype=np.uint32)
    pad[:, :n] = b
    return (pad.reshape(F, W, 32) << np.arange(32, dtype=np.uint32)).sum(axis=2).astype(np.uint32)


class _ServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("arena_bytes", ctypes.c_int64),
                ("max_batch_frames", ctypes.c_int64), ("min_batch_frames", ctypes.c_int64),
                ("max_wait_us", ctypes.c_int64), ("fuse_codes", ctypes.c_int)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("frames_completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("latency_p50_us", ctypes.c_double), ("latency_p99_us", ctypes.c_double),
                ("latency_max_us", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("cancelled", ctypes.c_int64)]


def _load_server_api(lib):
    if getattr(lib, "_server_sigs", False):
        return lib
    V, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "rmdec_server_create": ([ctypes.POINTER(V), ctypes.POINTER(_ServerConfig)], I),
        "rmdec_server_add_decoder": ([V, V, ctypes.POINTER(I)], I),
        "rmdec_server_submit": ([V, I, V, I64, V, ctypes.POINTER(U64)], I),
        "rmdec_server_poll": ([V, U64, I64, ctypes.POINTER(D)], I),
        "rmdec_server_stats_get": ([V, ctypes.POINTER(_ServerStats)], I),
        "rmdec_server_cancel": ([V, U64], I),
        "rmdec_server_destroy": ([V], None),
        "rmdec_server_last_error": ([V], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    lib._server_sigs = True
    return lib


class Server:
    """Continuous-batching request server (include/rmdec_serve.h) over Decoder handles."""

    def __init__(self, n_streams=4, arena_bytes=1 << 30, max_batch_frames=1 << 16, min_batch_frames=0,
                 max_wait_us=0, fuse_codes=False):
        self._lib = _load_server_api(load_library())
        cfg = _ServerConfig(n_streams, arena_bytes, max_batch_frames, min_batch_frames, max_wait_us,
                            1 if fuse_codes else 0)
        h = ctypes.c_void_p()
        st = self._lib.rmdec_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != OK:
            raise RmdecError(st, self._lib.rmdec_server_last_error(None).decode())
        self._h = h
        self._decoders = []

    def _check(self, st):
        if st != OK:
            raise RmdecError(st, self._lib.rmdec_server_last_error(self._h).decode())

    def add_decoder(self, dec):
        cid = ctypes.c_int()
        self._check(self._lib.rmdec_server_add_decoder(self._h, dec._h, ctypes.byref(cid)))
        self._decoders.append(dec)  # keep the handle alive for the server's lifetime
        return cid.value

    def submit(self, code_id, llr_host, out_host):
        """llr_host / out_host: CPU tensors (pinned for speed) that outlive the request."""
        rid = ctypes.c_uint64()
        self._check(self._lib.rmdec_server_submit(self._h, code_id, llr_host.data_ptr(), llr_host.shape[0],
                                                  out_host.data_ptr(), ctypes.byref(rid)))
        return rid.value

    def poll(self, request, timeout_us=0):
        """Returns (status, latency_us); status OK, EBUSY, ETIMEDOUT or ECANCELED (others raise)."""
        lat = ctypes.c_double(-1.0)
        st = self._lib.rmdec_server_poll(self._h, request, int(timeout_us), ctypes.byref(lat))
        if st in (OK, EBUSY, ETIMEDOUT, ECANCELED):
            return st, lat.value
        self._check(st)

    def cancel(self, request):
        """Cancels a request not yet admitted: returns True, or False if it was already admitted."""
        st = self._lib.rmdec_server_cancel(self._h, request)
        if st == EBUSY:
            return False
        self._check(st)
        return True

    def stats(self):
        s = _ServerStats()
        self._check(self._lib.rmdec_server_stats_get(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rmdec_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
