"""GB300 HERS encrypted search: Python binding of libhers.so (include/hers.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch provides device memory (uint64 data is held in int64
tensors, bit for bit) and streams.  There is no CPU fallback: if the library
is missing this module raises on import of the library (`lib()`), and the
functions raise HersError on any non-zero status.

The functions keep the C names:
  hers_keygen, hers_encrypt_gallery, hers_encrypt_probe, hers_probe_prepare,
  hers_search, hers_search_host, hers_decrypt_scores, hers_keys_export, ...
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
import weakref

N = 4096
MAX_D = 512
HERS_OK = 0
HERS_E_TIMEOUT = -4
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhers.so")

_lock = threading.Lock()
_lib = None


class HersError(RuntimeError):
    pass


# Live handles (contexts, keys, batches, servers), oldest first.  At
# interpreter exit they are closed newest first, while the CUDA runtime and
# this module are still whole, so a program that leaves them to the garbage
# collector ends the same way as one that closes them.
_live = []


def _register(obj):
    with _lock:
        _live[:] = [r for r in _live if r() is not None]
        _live.append(weakref.ref(obj))


@atexit.register
def _close_live_handles():
    for r in reversed(_live):
        obj = r()
        if obj is not None:
            try:
                obj.close()
            except Exception:
                pass
    _live.clear()


def build_library(force: bool = False) -> str:
    """Compile libhers.so in-tree with nvcc (sm_103a)."""
    from .build import build as _build
    return _build(force=force)


def lib():
    """The loaded libhers.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise HersError(f"{LIB_PATH} is missing: build it with "
                                "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            sigs = {
                "hers_default_params": ([vp], i32),
                "hers_create": ([vp, i32, vp], i32),
                "hers_destroy": ([vp], i32),
                "hers_last_error": ([vp], ctypes.c_char_p),
                "hers_status_string": ([i32], ctypes.c_char_p),
                "hers_ct_bytes": ([], u64),
                "hers_gallery_bytes": ([u64, u32], u64),
                "hers_probe_bytes": ([u32], u64),
                "hers_search_workspace_bytes": ([u64], u64),
                "hers_search_host_workspace_bytes": ([u64, u32], u64),
                "hers_blocks_for": ([u64], u64),
                "hers_keygen": ([vp, u64, vp], i32),
                "hers_keys_free": ([vp], i32),
                "hers_keys_export": ([vp, vp, vp, vp, vp], i32),
                "hers_encrypt_gallery": ([vp, vp, vp, u64, u32, u64, vp, vp, vp], i32),
                "hers_encrypt_probe": ([vp, vp, vp, u32, u64, vp, vp], i32),
                "hers_probe_prepare": ([vp, vp, u32, vp, vp], i32),
                "hers_search": ([vp, vp, vp, u64, u32, vp, vp, vp, u64, vp], i32),
                "hers_search_rerand": ([vp, vp, vp, u64, u32, vp, vp, vp, u64, u64, vp], i32),
                "hers_basew_digits": ([u32], u32),
                "hers_keys_add_basew": ([vp, vp, u64, u32], i32),
                "hers_keys_export_basew": ([vp, vp, vp], i32),
                "hers_search_basew": ([vp, vp, vp, u64, u32, vp, vp, vp, u64, vp], i32),
                "hers_search_host": ([vp, vp, vp, u64, u32, vp, vp, vp, u64, vp], i32),
                "hers_search_host_async": ([vp, vp, vp, u64, u32, vp, vp, vp, u64, vp], i32),
                "hers_search_noalloc": ([vp, vp, vp, u64, u32, vp, vp, vp], i32),
                "hers_decrypt_scores": ([vp, vp, vp, u64, vp, u64, vp], i32),
                "hers_check": ([vp, vp], i32),
                "hers_trace_enable": ([vp, u32], i32),
                "hers_trace_read": ([vp, vp, vp], i32),
                "hers_kernel_launches": ([], u64),
                "hers_probe_int_pipe": ([i32, u32, u64, vp], i32),
                "hers_selftest_wait_timeout": ([vp, u64, vp], i32),
                "hers_topk_workspace_bytes": ([u64], u64),
                "hers_enroll_workspace_bytes": ([u32], u64),
                "hers_enroll": ([vp, vp, vp, u64, u32, u64, u32, vp, u64, vp, u64, vp], i32),
                "hers_topk": ([vp, vp, u64, u32, vp, vp, vp, u64, vp], i32),
                "hers_tensor_variants": ([], i32),
                "hers_tensor_variant_name": ([i32], ctypes.c_char_p),
                "hers_get_tensor_variant": ([vp], i32),
                "hers_set_tensor_variant": ([vp, i32], i32),
                "hers_autotune": ([vp, vp, vp, u64, u32, vp, vp, u64, vp, vp, vp], i32),
                "hers_batch_workspace_bytes": ([vp, u32], u64),
                "hers_batch_create": ([vp, vp, vp, u32, vp, vp, u64, u32, vp], i32),
                "hers_batch_run": ([vp, vp], i32),
                "hers_batch_info": ([vp, vp, vp, vp, vp, vp], i32),
                "hers_batch_free": ([vp], i32),
                "hers_batch_trace": ([vp, vp, vp, vp], i32),
                "hers_search_stream_workspace_bytes": ([u32, u32, u32], u64),
                "hers_search_stream": ([vp, vp, vp, i32, u64, u32, vp, u32, vp, u32, i32, vp, u64,
                                        vp], i32),
                "hers_server_create": ([vp, vp, vp, u32, u64, u32, i32, vp], i32),
                "hers_server_submit": ([vp, u32, u64, u64, vp, vp, vp], i32),
                "hers_server_wait": ([vp, u64, u32, vp], i32),
                "hers_server_stats": ([vp, vp, vp, vp, vp, vp, vp], i32),
                "hers_server_pause": ([vp, i32], i32),
                "hers_server_free": ([vp], i32),
                "hers_server_timing": ([vp, vp, vp, vp], i32),
                "hers_set_tensor_first": ([vp, i32], i32),
                "hers_get_tensor_first": ([vp], i32),
                "hers_autotune_extension": ([vp, u32, vp, vp, vp], i32),
                "hers_epilogue_variants": ([], i32),
                "hers_epilogue_variant_name": ([i32], ctypes.c_char_p),
                "hers_get_epilogue_variant": ([vp], i32),
                "hers_set_epilogue_variant": ([vp, i32], i32),
                "hers_autotune_epilogue": ([vp, vp, vp, u64, u32, vp, vp, u64, vp, vp, vp], i32),
                "hers_batch_variants": ([], i32),
                "hers_batch_variant_name": ([i32], ctypes.c_char_p),
                "hers_keys_import": ([vp, vp, vp, vp], i32),
                "hers_keys_has_secret": ([vp], i32),
                "hers_search_range": ([vp, vp, vp, u64, u32, u64, u64, vp, vp, vp, u64, vp], i32),
                "hers_encrypt_gallery_host": ([vp, vp, vp, u64, u32, u64, vp, vp, vp], i32),
                "hers_decrypt_scores_host": ([vp, vp, vp, u64, vp, u64], i32),
                "hers_export_ct": ([vp, vp, u64, u32, u64, u64, vp], i32),
                "hers_import_ct": ([vp, vp, u64, u32, u64, u64, vp], i32),
            }
            for name, (args, res) in sigs.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class HersParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("q", ctypes.c_uint64 * 2), ("t", ctypes.c_uint64),
                ("flags", ctypes.c_uint32)]


T_DEFAULT = 4169729
T_PAPER = 1032193


class Context:
    """A library context on one CUDA device (hers_create / hers_destroy).
    t: the plaintext modulus, T_DEFAULT or the paper's T_PAPER."""

    def __init__(self, device: int = 0, t: int = None):
        self.device = device
        h = ctypes.c_void_p()
        params = None
        if t is not None:
            params = HersParams()
            lib().hers_default_params(ctypes.byref(params))
            params.t = t
            params = ctypes.byref(params)
        rc = lib().hers_create(params, device, ctypes.byref(h))
        if rc != HERS_OK:
            raise HersError(f"hers_create: {lib().hers_status_string(rc).decode()}")
        self.h = h
        _register(self)

    def check(self, rc, what):
        if rc != HERS_OK:
            msg = lib().hers_last_error(self.h).decode()
            raise HersError(f"{what}: {lib().hers_status_string(rc).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            lib().hers_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Keys:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        _register(self)

    def close(self):
        if getattr(self, "h", None):
            lib().hers_keys_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ sizes

def hers_ct_bytes():
    return int(lib().hers_ct_bytes())


def hers_blocks_for(m):
    return int(lib().hers_blocks_for(m))


def hers_gallery_bytes(nblocks, d):
    return int(lib().hers_gallery_bytes(nblocks, d))


def hers_probe_bytes(d):
    return int(lib().hers_probe_bytes(d))


def hers_search_workspace_bytes(nblocks):
    return int(lib().hers_search_workspace_bytes(nblocks))


def hers_search_host_workspace_bytes(nblocks, d):
    return int(lib().hers_search_host_workspace_bytes(nblocks, d))


def _words(nbytes, device):
    import torch
    return torch.empty(nbytes // 8, dtype=torch.int64, device=device)


# ------------------------------------------------------------------ scheme

def hers_keygen(ctx: Context, seed: int) -> Keys:
    h = ctypes.c_void_p()
    ctx.check(lib().hers_keygen(ctx.h, seed, ctypes.byref(h)), "hers_keygen")
    return Keys(ctx, h)


def hers_keys_export(ctx: Context, keys: Keys):
    """(sk int8[N], pk uint64[2,2,N], evk uint64[2,2,2,N]) as numpy arrays."""
    import numpy as np
    sk = np.zeros(N, dtype=np.int8)
    pk = np.zeros((2, 2, N), dtype=np.uint64)
    evk = np.zeros((2, 2, 2, N), dtype=np.uint64)
    ctx.check(lib().hers_keys_export(ctx.h, keys.h, sk.ctypes.data, pk.ctypes.data,
                                     evk.ctypes.data), "hers_keys_export")
    return sk, pk, evk


def hers_keys_import(ctx: Context, pk, evk) -> Keys:
    """A server-side key handle from the client's canonical pk [2,2,N] and
    evk [2,2,2,N] (uint64 numpy arrays, as hers_keys_export returns them):
    no secret key on it."""
    import numpy as np
    pk = np.ascontiguousarray(pk, dtype=np.uint64)
    evk = np.ascontiguousarray(evk, dtype=np.uint64)
    assert pk.shape == (2, 2, N) and evk.shape == (2, 2, 2, N)
    h = ctypes.c_void_p()
    ctx.check(lib().hers_keys_import(ctx.h, pk.ctypes.data, evk.ctypes.data, ctypes.byref(h)),
              "hers_keys_import")
    return Keys(ctx, h)


def hers_keys_has_secret(keys: Keys) -> bool:
    return bool(lib().hers_keys_has_secret(keys.h))


def hers_encrypt_gallery_host(ctx: Context, keys: Keys, feats, seed: int, want_ct: bool = False,
                              resident: bool = True, device=None, stream=None):
    """feats: host int8 [m, d] (numpy).  Returns (resident gallery words or
    None, canonical cts [nb,d,2,2,N] or None), on `device` (default: the
    context's CUDA device)."""
    import numpy as np
    import torch
    feats = np.ascontiguousarray(feats, dtype=np.int8)
    assert feats.ndim == 2
    m, d = feats.shape
    nb = hers_blocks_for(m)
    dev = device if device is not None else torch.device("cuda", ctx.device)
    want_ct = want_ct or not resident
    gal = _words(hers_gallery_bytes(nb, d), dev) if resident else None
    cts = torch.empty((nb, d, 2, 2, N), dtype=torch.int64, device=dev) if want_ct else None
    ctx.check(lib().hers_encrypt_gallery_host(ctx.h, keys.h, feats.ctypes.data, m, d, seed, _ptr(gal),
                                              _ptr(cts), _stream(stream)), "hers_encrypt_gallery_host")
    return gal, cts


def hers_export_ct(ctx: Context, gallery, nblocks: int, d: int, begin: int = 0, end: int = None):
    """Canonical cts of resident blocks [begin, end) as numpy uint64 [end-begin, d, 2, 2, N]."""
    import numpy as np
    end = nblocks if end is None else end
    out = np.zeros((max(0, end - begin), d, 2, 2, N), dtype=np.uint64)
    ctx.check(lib().hers_export_ct(ctx.h, _ptr(gallery), nblocks, d, begin, end, out.ctypes.data),
              "hers_export_ct")
    return out


def hers_import_ct(ctx: Context, ct_host, gallery, nblocks: int, d: int, begin: int = 0):
    """Canonical cts (numpy uint64 [k, d, 2, 2, N]) into resident blocks [begin, begin + k)."""
    import numpy as np
    ct_host = np.ascontiguousarray(ct_host, dtype=np.uint64)
    k = ct_host.shape[0]
    ctx.check(lib().hers_import_ct(ctx.h, ct_host.ctypes.data, nblocks, d, begin, begin + k, _ptr(gallery)),
              "hers_import_ct")
    return gallery


def hers_encrypt_gallery(ctx: Context, keys: Keys, feats, seed: int, want_ct: bool = False,
                         out=None, out_ct=None, stream=None, resident: bool = True):
    """feats: cuda int8 [m, d].  Returns (resident gallery words or None,
    canonical cts [nb,d,2,2,N] or None).  resident=False writes only the
    canonical cts (for hers_search_stream)."""
    import torch
    assert feats.is_cuda and feats.dtype == torch.int8 and feats.dim() == 2
    feats = feats.contiguous()
    m, d = feats.shape
    nb = hers_blocks_for(m)
    want_ct = want_ct or not resident
    gal = None
    if resident:
        gal = out if out is not None else _words(hers_gallery_bytes(nb, d), feats.device)
    cts = out_ct
    if want_ct and cts is None:
        cts = torch.empty((nb, d, 2, 2, N), dtype=torch.int64, device=feats.device)
    ctx.check(lib().hers_encrypt_gallery(ctx.h, keys.h, _ptr(feats), m, d, seed, _ptr(gal),
                                         _ptr(cts), _stream(stream)), "hers_encrypt_gallery")
    return gal, cts


def hers_encrypt_probe(ctx: Context, keys: Keys, q, seed: int, out=None, stream=None):
    """q: cuda int8 [d].  Returns canonical probe cts [d, 2, 2, N] (int64 view of uint64)."""
    import torch
    assert q.is_cuda and q.dtype == torch.int8 and q.dim() == 1
    q = q.contiguous()
    d = q.shape[0]
    cts = out if out is not None else torch.empty((d, 2, 2, N), dtype=torch.int64, device=q.device)
    ctx.check(lib().hers_encrypt_probe(ctx.h, keys.h, _ptr(q), d, seed, _ptr(cts), _stream(stream)),
              "hers_encrypt_probe")
    return cts


def hers_probe_prepare(ctx: Context, probe_ct, out=None, stream=None):
    d = probe_ct.shape[0]
    pr = out if out is not None else _words(hers_probe_bytes(d), probe_ct.device)
    ctx.check(lib().hers_probe_prepare(ctx.h, _ptr(probe_ct), d, _ptr(pr), _stream(stream)),
              "hers_probe_prepare")
    return pr


def hers_search(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe, out=None,
                workspace=None, stream=None):
    """Score cts [nblocks, 2, 2, N] (int64 view) of one prepared probe."""
    import torch
    dev = gallery.device
    sc = out if out is not None else torch.empty((nblocks, 2, 2, N), dtype=torch.int64, device=dev)
    wsb = hers_search_workspace_bytes(nblocks)
    ws = workspace if workspace is not None else _words(wsb, dev)
    ctx.check(lib().hers_search(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe), _ptr(sc),
                                _ptr(ws), ws.numel() * 8, _stream(stream)), "hers_search")
    return sc


def hers_keys_add_basew(ctx: Context, keys: Keys, seed: int, logw: int):
    """Attach base-w evaluation keys (w = 2^logw) to `keys`."""
    ctx.check(lib().hers_keys_add_basew(ctx.h, keys.h, seed, logw), "hers_keys_add_basew")


def hers_keys_export_basew(ctx: Context, keys: Keys, logw: int):
    """The base-w evaluation keys, uint64 [l][2][2][N] (canonical)."""
    import numpy as np
    out = np.zeros((int(lib().hers_basew_digits(logw)), 2, 2, N), dtype=np.uint64)
    ctx.check(lib().hers_keys_export_basew(ctx.h, keys.h, out.ctypes.data), "hers_keys_export_basew")
    return out


def hers_search_basew(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe, out=None,
                      workspace=None, stream=None):
    """hers_search with the base-w gadget for the key switch."""
    import torch
    dev = gallery.device
    sc = out if out is not None else torch.empty((nblocks, 2, 2, N), dtype=torch.int64, device=dev)
    ws = workspace if workspace is not None else _words(hers_search_workspace_bytes(nblocks), dev)
    ctx.check(lib().hers_search_basew(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe), _ptr(sc),
                                      _ptr(ws), ws.numel() * 8, _stream(stream)), "hers_search_basew")
    return sc


def hers_search_rerand(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe, rerand_seed: int,
                       out=None, workspace=None, stream=None):
    """hers_search plus a fresh Enc(0) (streams (rerand_seed, 0x31.., block)) on every block."""
    import torch
    dev = probe.device
    if out is None:
        out = torch.empty((nblocks, 2, 2, N), dtype=torch.int64, device=dev)
    if workspace is None:
        workspace = _words(int(lib().hers_search_workspace_bytes(nblocks)), dev)
    ctx.check(lib().hers_search_rerand(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe), _ptr(out),
                                       _ptr(workspace), workspace.numel() * 8, rerand_seed, _stream(stream)),
              "hers_search_rerand")
    return out


def hers_search_host(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe_ct_host,
                     scores_host, workspace, stream=None):
    """probe_ct_host / scores_host: CPU tensors (ideally pinned) of int64 words."""
    ctx.check(lib().hers_search_host(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe_ct_host),
                                     _ptr(scores_host), _ptr(workspace), workspace.numel() * 8,
                                     _stream(stream)), "hers_search_host")
    return scores_host


def hers_search_host_async(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe_ct_host,
                           scores_host, workspace, stream=None):
    """hers_search_host enqueued on `stream` without waiting: probe_ct_host and
    scores_host must be pinned CPU tensors; synchronise `stream` before reading
    scores_host or reusing the buffers or the workspace."""
    ctx.check(lib().hers_search_host_async(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe_ct_host),
                                           _ptr(scores_host), _ptr(workspace), workspace.numel() * 8,
                                           _stream(stream)), "hers_search_host_async")
    return scores_host


def hers_search_stream(ctx: Context, keys: Keys, gallery_ct, nblocks: int, d: int, probes,
                       chunk_blocks: int = 32, variant: int = 1, out=None, workspace=None,
                       stream=None):
    """Streamed search of a canonical gallery (CPU tensor: from host memory; CUDA
    tensor: from device memory) with several prepared probes.  Returns score
    cts [nprobes, nblocks, 2, 2, N] (int64 view) on the probes' device."""
    import torch
    dev = probes[0].device
    on_host = not gallery_ct.is_cuda
    np_ = len(probes)
    sc = out if out is not None else torch.empty((np_, nblocks, 2, 2, N), dtype=torch.int64,
                                                 device=dev)
    wsb = int(lib().hers_search_stream_workspace_bytes(d, np_, chunk_blocks))
    ws = workspace if workspace is not None else _words(wsb, dev)
    ptrs = (ctypes.c_void_p * np_)(*[p.data_ptr() for p in probes])
    ctx.check(lib().hers_search_stream(ctx.h, keys.h, _ptr(gallery_ct), 1 if on_host else 0,
                                       nblocks, d, ptrs, np_, _ptr(sc), chunk_blocks, variant,
                                       _ptr(ws), ws.numel() * 8, _stream(stream)),
              "hers_search_stream")
    return sc


def hers_search_stream_workspace_bytes(d, nprobes, chunk_blocks):
    return int(lib().hers_search_stream_workspace_bytes(d, nprobes, chunk_blocks))


def hers_decrypt_scores(ctx: Context, keys: Keys, scores_ct, m: int, out=None, stream=None):
    """int32 [m] decrypted, decoded scores (cuda)."""
    import torch
    nb = scores_ct.shape[0]
    out = out if out is not None else torch.empty(m, dtype=torch.int32, device=scores_ct.device)
    ctx.check(lib().hers_decrypt_scores(ctx.h, keys.h, _ptr(scores_ct), nb, _ptr(out), m,
                                        _stream(stream)), "hers_decrypt_scores")
    return out


def hers_decrypt_scores_host(ctx: Context, keys: Keys, scores_ct_host, m: int):
    """int32 [m] scores (numpy) from host score cts [nb, 2, 2, N] (int64 or uint64)."""
    import numpy as np
    import torch
    if isinstance(scores_ct_host, torch.Tensor):
        scores_ct_host = scores_ct_host.numpy()
    cts = np.ascontiguousarray(scores_ct_host).view(np.uint64)
    nb = cts.shape[0]
    out = np.zeros(m, dtype=np.int32)
    ctx.check(lib().hers_decrypt_scores_host(ctx.h, keys.h, cts.ctypes.data, nb, out.ctypes.data, m),
              "hers_decrypt_scores_host")
    return out


def hers_search_range(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, begin: int, end: int, probe,
                      out=None, workspace=None, stream=None):
    """Score cts [end - begin, 2, 2, N] of blocks [begin, end) of a resident gallery."""
    import torch
    dev = gallery.device
    n = max(0, end - begin)
    # an empty range still passes non-null buffers (the call checks them)
    sc = out if out is not None else torch.empty((max(n, 1), 2, 2, N), dtype=torch.int64, device=dev)
    ws = workspace if workspace is not None else _words(max(8, hers_search_workspace_bytes(n)), dev)
    ctx.check(lib().hers_search_range(ctx.h, keys.h, _ptr(gallery), nblocks, d, begin, end, _ptr(probe),
                                      _ptr(sc), _ptr(ws), ws.numel() * 8, _stream(stream)), "hers_search_range")
    return sc[:n]


def hers_check(ctx: Context, stream=None):
    ctx.check(lib().hers_check(ctx.h, _stream(stream)), "hers_check")


TRACE_PHASES = ("tensor", "intt", "scale_round", "key_switch", "search")


def hers_trace_enable(ctx: Context, max_calls: int):
    ctx.check(lib().hers_trace_enable(ctx.h, max_calls), "hers_trace_enable")


def hers_trace_read(ctx: Context):
    """(ncalls, {phase: average ms}) of the traced search calls since enabling."""
    n = ctypes.c_uint32()
    avg = (ctypes.c_double * len(TRACE_PHASES))()
    ctx.check(lib().hers_trace_read(ctx.h, ctypes.byref(n), avg), "hers_trace_read")
    return int(n.value), dict(zip(TRACE_PHASES, list(avg)))


def hers_kernel_launches():
    return int(lib().hers_kernel_launches())


def hers_tensor_variants():
    """Names of the tensor-kernel shapes, by index."""
    L = lib()
    return [L.hers_tensor_variant_name(i).decode() for i in range(L.hers_tensor_variants())]


def hers_get_tensor_variant(ctx: Context) -> int:
    return int(lib().hers_get_tensor_variant(ctx.h))


def hers_set_tensor_variant(ctx: Context, v: int):
    ctx.check(lib().hers_set_tensor_variant(ctx.h, v), "hers_set_tensor_variant")


def hers_set_tensor_first(ctx: Context, on: bool):
    ctx.check(lib().hers_set_tensor_first(ctx.h, 1 if on else 0), "hers_set_tensor_first")


def hers_get_tensor_first(ctx: Context) -> bool:
    return bool(lib().hers_get_tensor_first(ctx.h))


def hers_autotune_extension(ctx: Context, d: int, stream=None):
    """(cluster form chosen, {"per_polynomial": ms, "cluster": ms}) for preparing a probe of dimension d."""
    cl = ctypes.c_int()
    ms = (ctypes.c_double * 2)()
    ctx.check(lib().hers_autotune_extension(ctx.h, d, _stream(stream), ctypes.byref(cl), ms),
              "hers_autotune_extension")
    return bool(cl.value), {"per_polynomial": ms[0], "cluster": ms[1]}


def hers_epilogue_variants():
    L = lib()
    return [L.hers_epilogue_variant_name(v).decode() for v in range(L.hers_epilogue_variants())]


def hers_get_epilogue_variant(ctx: Context) -> int:
    return int(lib().hers_get_epilogue_variant(ctx.h))


def hers_set_epilogue_variant(ctx: Context, v: int):
    ctx.check(lib().hers_set_epilogue_variant(ctx.h, v), "hers_set_epilogue_variant")


def hers_autotune_epilogue(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe, workspace=None,
                           stream=None):
    """(chosen epilogue form, {name: ms}) for this search; the context keeps the fastest form."""
    names = hers_epilogue_variants()
    ws = workspace if workspace is not None else _words(hers_search_workspace_bytes(nblocks), gallery.device)
    chosen = ctypes.c_int()
    ms = (ctypes.c_double * len(names))()
    ctx.check(lib().hers_autotune_epilogue(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe), _ptr(ws),
                                           ws.numel() * 8, _stream(stream), ctypes.byref(chosen), ms),
              "hers_autotune_epilogue")
    return chosen.value, {names[i]: ms[i] for i in range(len(names))}


def hers_autotune(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, probe, workspace=None,
                  stream=None):
    """Times every tensor-kernel shape on this search, keeps the fastest on ctx.
    Returns (chosen index, {name: ms})."""
    names = hers_tensor_variants()
    ws = workspace if workspace is not None else _words(hers_search_workspace_bytes(nblocks),
                                                        gallery.device)
    chosen = ctypes.c_int()
    ms = (ctypes.c_double * len(names))()
    ctx.check(lib().hers_autotune(ctx.h, keys.h, _ptr(gallery), nblocks, d, _ptr(probe), _ptr(ws),
                                  ws.numel() * 8, _stream(stream), ctypes.byref(chosen), ms),
              "hers_autotune")
    return int(chosen.value), dict(zip(names, list(ms)))


class BatchItem(ctypes.Structure):
    _fields_ = [("gallery", ctypes.c_void_p), ("nblocks", ctypes.c_uint64), ("d", ctypes.c_uint32),
                ("probe", ctypes.c_void_p)]


BATCH_AUTOTUNE = 1


def batch_variant_flag(v: int) -> int:
    return (v + 1) << 8


def hers_batch_variants():
    L = lib()
    return [L.hers_batch_variant_name(i).decode() for i in range(L.hers_batch_variants())]


class Batch:
    """A planned, graph-captured batched search (hers_batch_create / run / free).

    items: list of (gallery tensor, nblocks, d, prepared probe tensor).
    Score ciphertexts of item i are rows [off_i, off_i + nblocks_i) of .scores,
    off_i = sum of the previous items' nblocks.
    """

    def __init__(self, ctx: Context, keys: Keys, items, flags: int = BATCH_AUTOTUNE):
        import torch
        self.ctx, self.keys = ctx, keys
        self._keep = [(g, p) for g, _, _, p in items]  # the plan points into these
        arr = (BatchItem * len(items))()
        for i, (g, nb, d, p) in enumerate(items):
            arr[i] = BatchItem(g.data_ptr(), nb, d, p.data_ptr())
        self._items = arr
        self.offsets = []
        off = 0
        for _, nb, _, _ in items:
            self.offsets.append(off)
            off += nb
        self.npairs = off
        dev = items[0][0].device
        self.scores = torch.empty((off, 2, 2, N), dtype=torch.int64, device=dev)
        wsb = int(lib().hers_batch_workspace_bytes(arr, len(items)))
        self.workspace = _words(wsb, dev)
        h = ctypes.c_void_p()
        torch.cuda.synchronize(dev)
        ctx.check(lib().hers_batch_create(ctx.h, keys.h, arr, len(items), _ptr(self.scores),
                                          _ptr(self.workspace), wsb, flags, ctypes.byref(h)),
                  "hers_batch_create")
        self.h = h
        _register(self)

    def run(self, stream=None):
        self.ctx.check(lib().hers_batch_run(self.h, _stream(stream)), "hers_batch_run")
        return self.scores

    def info(self):
        v, ng, nu, npairs = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        names = hers_batch_variants()
        tm = (ctypes.c_double * len(names))()
        lib().hers_batch_info(self.h, ctypes.byref(v), ctypes.byref(ng), ctypes.byref(nu),
                              ctypes.byref(npairs), tm)
        return {"variant": names[v.value], "groups": ng.value, "units": nu.value,
                "pairs": npairs.value, "tune_ms": {n: t for n, t in zip(names, list(tm)) if t >= 0}}

    def trace(self, stream=None):
        """One traced run (same launches, outside the graph): (tensor ms, whole run ms)."""
        t, a = ctypes.c_double(), ctypes.c_double()
        self.ctx.check(lib().hers_batch_trace(self.h, _stream(stream), ctypes.byref(t),
                                              ctypes.byref(a)), "hers_batch_trace")
        return t.value, a.value

    def item_scores(self, i, nblocks):
        return self.scores[self.offsets[i]: self.offsets[i] + nblocks]

    def close(self):
        if getattr(self, "h", None):
            lib().hers_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServerGallery(ctypes.Structure):
    _fields_ = [("gallery", ctypes.c_void_p), ("nblocks", ctypes.c_uint64), ("d", ctypes.c_uint32)]


class Server:
    """Continuous-batching server (hers_server_*).

    galleries: list of (resident gallery tensor, nblocks, d).  submit() takes
    the probe's canonical cts and an output buffer as CPU tensors (pinned for
    speed) which must stay alive until wait() returns for that id.
    """

    def __init__(self, ctx: Context, keys: Keys, galleries, workspace_bytes=0, max_batch=16,
                 variant=1):
        self.ctx, self.keys = ctx, keys  # the server uses both until it is closed
        self._keep = [g for g, _, _ in galleries]
        arr = (ServerGallery * len(galleries))()
        for i, (g, nb, d) in enumerate(galleries):
            arr[i] = ServerGallery(g.data_ptr(), nb, d)
        h = ctypes.c_void_p()
        ctx.check(lib().hers_server_create(ctx.h, keys.h, arr, len(galleries), workspace_bytes,
                                           max_batch, variant, ctypes.byref(h)), "hers_server_create")
        self.h = h
        _register(self)
        self._bufs = {}

    def submit(self, gallery: int, begin: int, end: int, probe_ct_host, scores_host) -> int:
        rid = ctypes.c_uint64()
        self.ctx.check(lib().hers_server_submit(self.h, gallery, begin, end, _ptr(probe_ct_host),
                                                _ptr(scores_host), ctypes.byref(rid)),
                       "hers_server_submit")
        self._bufs[rid.value] = (probe_ct_host, scores_host)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 600000):
        """(status, latency ms)."""
        lat = ctypes.c_double()
        rc = lib().hers_server_wait(self.h, rid, timeout_ms, ctypes.byref(lat))
        if rc != -4:
            self._bufs.pop(rid, None)
        return rc, lat.value

    def pause(self, paused: bool = True):
        self.ctx.check(lib().hers_server_pause(self.h, 1 if paused else 0), "hers_server_pause")

    def stats(self):
        v = [ctypes.c_uint64() for _ in range(6)]
        rc = lib().hers_server_stats(self.h, *[ctypes.byref(x) for x in v])
        keys = ("submitted", "completed", "batches", "entries", "max_batch_seen", "pool_bytes")
        out = dict(zip(keys, [x.value for x in v]))
        out["status"] = rc
        return out

    def timing(self):
        """Summed ms over finished batches: kernels and copies (device), plan (host)."""
        v = [ctypes.c_double() for _ in range(3)]
        self.ctx.check(lib().hers_server_timing(self.h, *[ctypes.byref(x) for x in v]), "hers_server_timing")
        return dict(zip(("kernels_ms", "copies_ms", "plan_ms"), [x.value for x in v]))

    def close(self):
        if getattr(self, "h", None):
            lib().hers_server_free(self.h)
            self.h = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


INT_PIPE_OPS = ("imad_wide_u32", "imad_u32", "umul64hi", "mad_wide_s32_outer")


def hers_probe_int_pipe(device: int = 0, iters: int = 1 << 16):
    """{op name: operations per second} of the integer pipes on `device`."""
    out = {}
    for i, name in enumerate(INT_PIPE_OPS):
        v = ctypes.c_double()
        rc = lib().hers_probe_int_pipe(device, i, iters, ctypes.byref(v))
        if rc != HERS_OK:
            raise HersError(f"hers_probe_int_pipe({name}): {lib().hers_status_string(rc).decode()}")
        out[name] = v.value
    return out


def hers_enroll(ctx: Context, keys: Keys, gallery, nblocks: int, d: int, block: int, slot: int, feats,
                seed: int, workspace=None, stream=None):
    """Online enrollment (Alg 6): int8 device features [d] into slot `slot` of
    resident block `block`; updates `gallery` in place."""
    import torch
    assert feats.is_cuda and feats.dtype == torch.int8 and feats.numel() == d
    feats = feats.contiguous()
    if workspace is None:
        workspace = _words(int(lib().hers_enroll_workspace_bytes(d)), feats.device)
    ctx.check(lib().hers_enroll(ctx.h, keys.h, _ptr(gallery), nblocks, d, block, slot, _ptr(feats), seed,
                                _ptr(workspace), workspace.numel() * 8, _stream(stream)), "hers_enroll")
    return gallery


def hers_topk(ctx: Context, scores, k: int, workspace=None, stream=None):
    """Stage-1 top-k of int32 device scores: (indices int64[k], scores int32[k]),
    score descending, ties by lowest index."""
    import torch
    assert scores.is_cuda and scores.dtype == torch.int32 and scores.dim() == 1
    m = scores.numel()
    if workspace is None:
        workspace = _words(int(lib().hers_topk_workspace_bytes(m)) + 7, scores.device)
    idx = torch.empty(k, dtype=torch.int64, device=scores.device)
    val = torch.empty(k, dtype=torch.int32, device=scores.device)
    ctx.check(lib().hers_topk(ctx.h, _ptr(scores), m, k, _ptr(idx), _ptr(val), _ptr(workspace),
                              workspace.numel() * 8, _stream(stream)), "hers_topk")
    return idx, val


def hers_selftest_wait_timeout(ctx: Context, limit_ns: int):
    """Runs the bounded-wait self-test: (status, kernel ms).  HERS_E_TIMEOUT is
    the expected status; this call does not raise on it."""
    ms = ctypes.c_double()
    rc = lib().hers_selftest_wait_timeout(ctx.h, limit_ns, ctypes.byref(ms))
    return rc, ms.value


def to_u64(t):
    """A device/host int64 tensor of ciphertext words as a numpy uint64 array."""
    return t.detach().cpu().numpy().view("uint64")
