"""HERS oracle: Python wrapper around oracle/hers_oracle.c.

TEST INFRASTRUCTURE ONLY.  A plain, slow, exact CPU implementation of the HERS
encrypted search (FV scheme of App. A, encoding of Sec. 3.2, Alg 7), used to
check the CUDA library bit for bit.  Only tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference legs may import it; the CUDA library never
does, and this package imports nothing from the library.

Exchange format (the same as the library's canonical form): a ciphertext is a
uint64 array [2 polys][2 limbs][n] of residues in [0, q1) and [0, q2).

Parity status: every function below is pinned by tests/test_oracle_pins.py
against closed forms, brute force or an independent library (see the pin
list in that file); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hers_oracle.c")
_HDR = os.path.join(_HERE, "cdt_table.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhers_oracle.so")

N = 4096
Q1 = 18014398509309953
Q2 = 18014398509293569
Q = Q1 * Q2
T = 4169729            # the default plaintext modulus
T_PAPER = 1032193      # the paper's (Sec. 4.1); select with set_plain_modulus
PURPOSE_GALLERY = 0x11  # u, e1, e2 streams at 0x11, 0x12, 0x13; obj = block * d + dim
PURPOSE_PROBE = 0x21    # u, e1, e2 streams at 0x21, 0x22, 0x23; obj = dim
PURPOSE_RERAND = 0x31   # output re-randomisation Enc(0): u, e1, e2 at 0x31..0x33; obj = block
PURPOSE_ENROLL = 0x41   # online enrollment (Alg 6): u, e1, e2 at 0x41..0x43; obj = (b n + v) d + dim

_lock = threading.Lock()
_lib = None


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("tensor_products", ctypes.c_uint64),
        ("tensor_adds", ctypes.c_uint64),
        ("scale_rounds", ctypes.c_uint64),
        ("key_switches", ctypes.c_uint64),
        ("rotations", ctypes.c_uint64),
        ("ties", ctypes.c_uint64),
        ("bound_violations", ctypes.c_uint64),
        ("max_x_bits", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/. Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i8p = ctypes.POINTER(ctypes.c_int8)
            c_int, c_u64, c_u32 = ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
            sp = ctypes.POINTER(OracleStats)
            L.orc_chacha20_block.argtypes = [u32p, c_u32, u32p, u32p]
            L.orc_sample.argtypes = [c_u64, c_u32, c_u64, c_int, c_int, c_u64, i64p]
            L.orc_negacyclic_z.argtypes = [c_int, i64p, i64p, u64p]
            L.orc_psi_t.argtypes = [c_int]
            L.orc_psi_t.restype = c_u64
            L.orc_encode.argtypes = [c_int, i64p, u32p]
            L.orc_decode.argtypes = [c_int, u32p, i64p]
            L.orc_keygen.argtypes = [c_int, c_u64, i8p, u64p, u64p]
            L.orc_encrypt.argtypes = [c_int, u64p, u32p, c_u64, c_u32, c_u64, u64p]
            L.orc_search_block.argtypes = [c_int, c_int, u64p, u64p, u64p, u64p, u64p, sp]
            L.orc_search_block_per_product.argtypes = [c_int, c_int, u64p, u64p, u64p, u64p,
                                                       u64p, sp]
            L.orc_decrypt.argtypes = [c_int, i8p, u64p, c_int, i64p, u32p, u64p]
            L.orc_params.argtypes = [u64p]
            L.orc_set_t.argtypes = [c_u64]
            L.orc_basew_digits.argtypes = [c_int]
            L.orc_keygen_w.argtypes = [c_int, c_u64, c_u64, c_int, u64p]
            L.orc_keyswitch_w.argtypes = [c_int, u64p, u64p, c_int, u64p]
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# --------------------------------------------------------------------------
# primitives exposed for pins
# --------------------------------------------------------------------------

def chacha20_block(key_words, counter, nonce_words):
    """The 16 output words of one ChaCha20 block (RFC 8439, Sec. 2.3)."""
    k = np.ascontiguousarray(key_words, dtype=np.uint32)
    nn = np.ascontiguousarray(nonce_words, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    lib().orc_chacha20_block(_p(k, ctypes.c_uint32), counter, _p(nn, ctypes.c_uint32),
                             _p(out, ctypes.c_uint32))
    return out


def sample(seed, purpose, obj, n, kind, qj=0):
    """kind 0: ternary, 1: chi (Gaussian), 2: uniform mod qj."""
    out = np.zeros(n, dtype=np.int64)
    _check(lib().orc_sample(seed, purpose, obj, n, kind, qj, _p(out, ctypes.c_int64)), "sample")
    return out


def negacyclic_z(a, b):
    """(a * b) mod (x^n + 1) over Z for integer lists |a_j|, |b_j| < 2^107."""
    n = len(a)
    aw = np.zeros(2 * n, dtype=np.int64)
    bw = np.zeros(2 * n, dtype=np.int64)
    mask = (1 << 64) - 1
    for j in range(n):
        for arr, v in ((aw, a[j]), (bw, b[j])):
            u = v & ((1 << 128) - 1)
            arr[2 * j] = np.uint64(u & mask).astype(np.int64)
            arr[2 * j + 1] = np.uint64(u >> 64).astype(np.int64)
    out = np.zeros(5 * n, dtype=np.uint64)
    _check(lib().orc_negacyclic_z(n, _p(aw, ctypes.c_int64), _p(bw, ctypes.c_int64),
                                  _p(out, ctypes.c_uint64)), "negacyclic_z")
    res = []
    for k in range(n):
        v = 0
        for w in range(5):
            v |= int(out[5 * k + w]) << (64 * w)
        if v >> 319:
            v -= 1 << 320
        res.append(v)
    return res


def psi_t(n=N):
    return int(lib().orc_psi_t(n))


# --------------------------------------------------------------------------
# scheme
# --------------------------------------------------------------------------

def encode(slots, n=N):
    s = np.ascontiguousarray(slots, dtype=np.int64)
    assert s.shape == (n,)
    m = np.zeros(n, dtype=np.uint32)
    _check(lib().orc_encode(n, _p(s, ctypes.c_int64), _p(m, ctypes.c_uint32)), "encode")
    return m


def decode(m, n=N):
    mm = np.ascontiguousarray(m, dtype=np.uint32)
    out = np.zeros(n, dtype=np.int64)
    _check(lib().orc_decode(n, _p(mm, ctypes.c_uint32), _p(out, ctypes.c_int64)), "decode")
    return out


def keygen(seed, n=N):
    """Alg 1. Returns (sk int8[n], pk uint64[2,2,n], evk uint64[2,2,2,n])."""
    sk = np.zeros(n, dtype=np.int8)
    pk = np.zeros((2, 2, n), dtype=np.uint64)
    evk = np.zeros((2, 2, 2, n), dtype=np.uint64)
    _check(lib().orc_keygen(n, seed, _p(sk, ctypes.c_int8), _p(pk, ctypes.c_uint64),
                            _p(evk, ctypes.c_uint64)), "keygen")
    return sk, pk, evk


def encrypt(pk, m, seed, purpose_base, obj, n=N):
    """Alg 2 on a plaintext m (uint32[n] in [0, t))."""
    pkc = np.ascontiguousarray(pk, dtype=np.uint64)
    mm = np.ascontiguousarray(m, dtype=np.uint32)
    ct = np.zeros((2, 2, n), dtype=np.uint64)
    _check(lib().orc_encrypt(n, _p(pkc, ctypes.c_uint64), _p(mm, ctypes.c_uint32), seed,
                             purpose_base, obj, _p(ct, ctypes.c_uint64)), "encrypt")
    return ct


def gallery_block_slots(feats, b, n=N):
    """Slots of the d gallery plaintexts of block b (Eq. 3): [d][n], slot j <- p_{bn+j}[i]."""
    m, d = feats.shape
    lo, hi = b * n, min((b + 1) * n, m)
    slots = np.zeros((d, n), dtype=np.int64)
    slots[:, : hi - lo] = feats[lo:hi, :].T.astype(np.int64)
    return slots


def encrypt_gallery_block(pk, feats, b, seed, n=N):
    """Ciphertexts [d][2][2][n] of gallery block b (Eq. 3 + Alg 2; obj = b*d + i)."""
    d = feats.shape[1]
    slots = gallery_block_slots(feats, b, n)
    out = np.zeros((d, 2, 2, n), dtype=np.uint64)
    for i in range(d):
        out[i] = encrypt(pk, encode(slots[i], n), seed, PURPOSE_GALLERY, b * d + i, n)
    return out


def encrypt_gallery_block_rows(pk, rows, b, seed, n=N):
    """Ciphertexts [d][2][2][n] of gallery block b given only that block's rows
    (rows[j] = entry b n + j; fewer than n rows pad with zeros)."""
    d = rows.shape[1]
    slots = np.zeros((d, n), dtype=np.int64)
    slots[:, : rows.shape[0]] = rows.T.astype(np.int64)
    out = np.zeros((d, 2, 2, n), dtype=np.uint64)
    for i in range(d):
        out[i] = encrypt(pk, encode(slots[i], n), seed, PURPOSE_GALLERY, b * d + i, n)
    return out


def encrypt_probe(pk, qfeat, seed, n=N):
    """Ciphertexts [d][2][2][n] of a probe (Eq. 2: dimension i in every slot; obj = i)."""
    d = len(qfeat)
    out = np.zeros((d, 2, 2, n), dtype=np.uint64)
    for i in range(d):
        m = encode(np.full(n, int(qfeat[i]), dtype=np.int64), n)
        out[i] = encrypt(pk, m, seed, PURPOSE_PROBE, i, n)
    return out


def search_block(probe_cts, gal_cts, evk, n=N, want_pre=False):
    """Score ciphertext of one block: accumulate over d, scale once, relinearise once."""
    d = probe_cts.shape[0]
    pc = np.ascontiguousarray(probe_cts, dtype=np.uint64)
    gc = np.ascontiguousarray(gal_cts, dtype=np.uint64)
    ev = np.ascontiguousarray(evk, dtype=np.uint64)
    out = np.zeros((2, 2, n), dtype=np.uint64)
    pre = np.zeros((3, 2, n), dtype=np.uint64)
    st = OracleStats()
    rc = lib().orc_search_block(n, d, _p(pc, ctypes.c_uint64), _p(gc, ctypes.c_uint64),
                                _p(ev, ctypes.c_uint64), _p(out, ctypes.c_uint64),
                                _p(pre, ctypes.c_uint64) if want_pre else None,
                                ctypes.byref(st))
    _check(rc, "search_block")
    return (out, pre, st.as_dict()) if want_pre else (out, st.as_dict())


def search_block_per_product(probe_cts, gal_cts, evk, init_ct=None, n=N):
    """Paper-literal Alg 7 inner loop with Alg 5 (scale + relinearise) per product."""
    d = probe_cts.shape[0]
    pc = np.ascontiguousarray(probe_cts, dtype=np.uint64)
    gc = np.ascontiguousarray(gal_cts, dtype=np.uint64)
    ev = np.ascontiguousarray(evk, dtype=np.uint64)
    out = np.zeros((2, 2, n), dtype=np.uint64)
    st = OracleStats()
    ini = None if init_ct is None else np.ascontiguousarray(init_ct, dtype=np.uint64)
    rc = lib().orc_search_block_per_product(n, d, _p(pc, ctypes.c_uint64),
                                            _p(gc, ctypes.c_uint64), _p(ev, ctypes.c_uint64),
                                            None if ini is None else _p(ini, ctypes.c_uint64),
                                            _p(out, ctypes.c_uint64), ctypes.byref(st))
    _check(rc, "search_block_per_product")
    return out, st.as_dict()


def decrypt(sk, ct, n=N):
    """Alg 3 + decode. ct: [2 or 3][2][n]. Returns (slots int64[n], pt uint32[n], max |noise|)."""
    c = np.ascontiguousarray(ct, dtype=np.uint64)
    ncomp = c.shape[0]
    s = np.ascontiguousarray(sk, dtype=np.int8)
    slots = np.zeros(n, dtype=np.int64)
    pt = np.zeros(n, dtype=np.uint32)
    noise = np.zeros(2, dtype=np.uint64)
    _check(lib().orc_decrypt(n, _p(s, ctypes.c_int8), _p(c, ctypes.c_uint64), ncomp,
                             _p(slots, ctypes.c_int64), _p(pt, ctypes.c_uint32),
                             _p(noise, ctypes.c_uint64)), "decrypt")
    return slots, pt, int(noise[0]) | (int(noise[1]) << 64)


def res_to_int(ct_poly_res):
    """[2 limbs][n] residues -> list of Python ints in [0, q) (CRT, for tests)."""
    r1, r2 = ct_poly_res
    inv = pow(Q1, -1, Q2)
    return [int(a) + Q1 * (((int(b) - int(a)) * inv) % Q2) for a, b in zip(r1, r2)]


def search_gallery(probe_cts, gal_blocks_cts, evk, n=N):
    """Score ciphertexts for a list of gallery blocks (Alg 7's outer loop)."""
    outs, tot = [], None
    for g in gal_blocks_cts:
        o, st = search_block(probe_cts, g, evk, n)
        outs.append(o)
        tot = st if tot is None else {k: tot[k] + st[k] for k in st}
    return np.stack(outs), tot


def topk(scores, k):
    """Stage 1 of the two-stage search (Sec. 3.2): the k gallery entries with
    the largest decrypted scores, ordered by score descending and, among equal
    scores, by index ascending.  Returns (indices int64[k], scores int32[k]).
    The plain definition: a stable sort of the indices by descending score."""
    s = np.asarray(scores)
    k = int(min(k, s.shape[0]))
    order = np.lexsort((np.arange(s.shape[0], dtype=np.int64), -s.astype(np.int64)))[:k]
    return order.astype(np.int64), s[order].astype(np.int32)


def ct_add(a, b):
    """Homomorphic addition (App. A): residue-wise sum of two canonical
    ciphertexts [2][2][n], mod q1 for limb 0 and q2 for limb 1."""
    out = np.empty_like(a)
    for l, q in enumerate((Q1, Q2)):
        out[:, l] = (a[:, l].astype(object) + b[:, l].astype(object)) % q
    return out.astype(np.uint64)


def rerandomize(pk, ct, seed, block, n=N):
    """Output re-randomisation (Alg 7 initialises s with Encrypt(0)): ct plus
    a fresh encryption of zero drawn from the streams (seed, 0x31.., block)."""
    zero = encrypt(pk, np.zeros(n, dtype=np.uint32), seed, PURPOSE_RERAND, block, n)
    return ct_add(ct, zero)


def enroll(pk, block_cts, b, v, feat, seed, n=N):
    """Online enrollment (Alg 6): adds one entry with features feat[d] into
    slot v of gallery block b.  For each dimension i: the plaintext with slot
    v = feat[i] and every other slot 0 (BatchEncode(.; v)), encrypted with the
    streams (seed, 0x41.., (b n + v) d + i), is added to the block's
    ciphertext i (CipherAdd).  block_cts: [d][2][2][n]; returns the updated copy."""
    d = block_cts.shape[0]
    out = np.empty_like(block_cts)
    for i in range(d):
        slots = np.zeros(n, dtype=np.int64)
        slots[v] = int(feat[i])
        z = encrypt(pk, encode(slots, n), seed, PURPOSE_ENROLL, (b * n + v) * d + i, n)
        out[i] = ct_add(block_cts[i], z)
    return out


def basew_digits(logw):
    """Digits l = ceil(bits(q) / logw) of the base-w gadget, w = 2^logw."""
    return int(lib().orc_basew_digits(logw))


def keygen_w(sk_seed, w_seed, logw, n=N):
    """Base-w evaluation keys (Alg 1 with g_j = w^j): [l][2][2][n]; s from
    sk_seed's secret-key stream, a_j / e_j from w_seed's streams 0x06 / 0x07."""
    evkw = np.zeros((basew_digits(logw), 2, 2, n), dtype=np.uint64)
    _check(lib().orc_keygen_w(n, sk_seed, w_seed, logw, _p(evkw, ctypes.c_uint64)), "keygen_w")
    return evkw


def keyswitch_w(ct3, evkw, logw, n=N):
    """Relinearisation of (c0, c1, c2) [3][2][n] with the base-w gadget."""
    c = np.ascontiguousarray(ct3, dtype=np.uint64)
    ev = np.ascontiguousarray(evkw, dtype=np.uint64)
    out = np.zeros((2, 2, n), dtype=np.uint64)
    _check(lib().orc_keyswitch_w(n, _p(c, ctypes.c_uint64), _p(ev, ctypes.c_uint64), logw,
                                 _p(out, ctypes.c_uint64)), "keyswitch_w")
    return out


def search_block_basew(probe_cts, gal_cts, evk, evkw, logw, n=N):
    """Score ciphertext of one block with the base-w gadget for the one key
    switch: the same tensor and scale-and-round as search_block."""
    _, pre, _ = search_block(probe_cts, gal_cts, evk, n, want_pre=True)
    return keyswitch_w(pre, evkw, logw, n)


def set_plain_modulus(t):
    """Selects the plaintext modulus for every later call: T (default) or
    T_PAPER.  Not for use while another thread calls the oracle."""
    _check(lib().orc_set_t(t), "set_plain_modulus")


def plain_modulus():
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_params(_p(out, ctypes.c_uint64))
    return int(out[2])
