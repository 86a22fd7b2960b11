"""Seeded synthetic inputs for HERS encrypted search.

This module is the only code shared by the oracle's tests and the CUDA
library's tests and benchmark.  It holds none of the method's arithmetic: it
only draws feature vectors shaped like the paper's workloads (Sec. 4: deep
features reduced to d in {32, 64, 128} dimensions, galleries of up to 100M
entries with planted mates) and quantises them to the int8 integers that both
sides take as input.

Recipe (stand-in for the paper's datasets, which are not used):
  gallery entry: x ~ N(0, I_d), x <- x / ||x||_2, p = clip(rint(127 x), -127, 127) as int8;
  probe of a mate: y = x_mate + n, n ~ N(0, (0.3 / sqrt(d))^2 I_d), y <- y / ||y||_2,
                   then quantised the same way;
  mates: distinct indices drawn without replacement.
Rows are generated in chunks of CHUNK entries from numpy's default_rng([seed, chunk]),
so any entry's float vector can be regenerated on its own.
"""
from __future__ import annotations

import numpy as np

CHUNK = 1 << 16        # entries per generator chunk (16 slot-packed blocks of 4096)
SCALE = 127            # int8 quantisation scale
PROBE_NOISE = 0.3      # total norm of the probe perturbation


def quantise(x: np.ndarray) -> np.ndarray:
    """L2-normalise rows and round to int8 at scale 127 (round half to even)."""
    nrm = np.linalg.norm(x, axis=-1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return np.clip(np.rint(SCALE * x / nrm), -SCALE, SCALE).astype(np.int8)


def _chunk_floats(seed: int, c: int, rows: int, d: int) -> np.ndarray:
    rng = np.random.default_rng([seed, c])
    return rng.standard_normal((rows, d))


def gallery_features(m: int, d: int, seed: int) -> np.ndarray:
    """int8 [m, d] gallery features."""
    out = np.empty((m, d), dtype=np.int8)
    for c in range((m + CHUNK - 1) // CHUNK):
        lo, hi = c * CHUNK, min((c + 1) * CHUNK, m)
        out[lo:hi] = quantise(_chunk_floats(seed, c, CHUNK, d)[: hi - lo])
    return out


def gallery_float_row(idx: int, d: int, seed: int) -> np.ndarray:
    """The unquantised float vector behind gallery entry idx."""
    c = idx // CHUNK
    return _chunk_floats(seed, c, CHUNK, d)[idx - c * CHUNK]


def mate_indices(m: int, count: int, seed: int) -> np.ndarray:
    """count distinct gallery indices in [0, m), in draw order."""
    rng = np.random.default_rng([seed, 0x6D617465])
    return rng.choice(m, size=count, replace=False).astype(np.int64)


def probe_for_mate(mate_idx: int, d: int, gallery_seed: int, probe_seed: int) -> np.ndarray:
    """int8 [d] probe: the mate's float vector plus N(0, (0.3/sqrt d)^2) noise, requantised."""
    x = gallery_float_row(mate_idx, d, gallery_seed)
    x = x / np.linalg.norm(x)
    rng = np.random.default_rng([probe_seed, int(mate_idx)])
    y = x + rng.standard_normal(d) * (PROBE_NOISE / np.sqrt(d))
    return quantise(y[None, :])[0]


def plain_inner_products(feats: np.ndarray, probe: np.ndarray) -> np.ndarray:
    """Eq. 1 in the clear, r = P^T q, as int64 (the value decrypted scores must equal)."""
    return feats.astype(np.int64) @ probe.astype(np.int64)


def gallery_features_device(m: int, d: int, seed: int, device, chunk: int = 1 << 22):
    """int8 [m, d] gallery features drawn on a CUDA device (torch's seeded
    generator): the same recipe as gallery_features, for galleries too large to
    draw on the host in reasonable time.  Deterministic for a given seed,
    device type and torch version; not bit-equal to gallery_features."""
    import torch
    out = torch.empty((m, d), dtype=torch.int8, device=device)
    for c in range((m + chunk - 1) // chunk):
        lo, hi = c * chunk, min((c + 1) * chunk, m)
        g = torch.Generator(device=device)
        g.manual_seed((seed * 1_000_003 + c) % (1 << 63))
        x = torch.randn((hi - lo, d), generator=g, device=device, dtype=torch.float32)
        x = x / x.norm(dim=1, keepdim=True).clamp_min(1e-12)
        out[lo:hi] = torch.round(SCALE * x).clamp_(-SCALE, SCALE).to(torch.int8)
    return out


def serving_requests(rate: float, window_s: float, max_requests: int, nblocks_total: int,
                     dims=(32, 64, 128), min_entries: int = 10_000, max_entries: int = 10_000_000,
                     seed: int = 0, n_block: int = 4096):
    """Poisson arrivals at `rate` per second over `window_s` seconds (at most
    max_requests).  Each request: arrival time, gallery index (its d drawn
    uniformly from dims), size uniform in [min_entries, max_entries] entries
    rounded up to whole blocks, and a uniform start block.  Returns a list of
    (t_arrival_s, gallery_index, block_begin, block_end)."""
    rng = np.random.default_rng([seed, 0x73657276])
    t, out = 0.0, []
    while len(out) < max_requests:
        t += rng.exponential(1.0 / rate)
        if t > window_s:
            break
        gi = int(rng.integers(0, len(dims)))
        size = int(rng.integers(min_entries, max_entries + 1))
        nb = min(nblocks_total, (size + n_block - 1) // n_block)
        b0 = int(rng.integers(0, nblocks_total - nb + 1))
        out.append((t, gi, b0, b0 + nb))
    return out


def batched_workload(total_blocks: int, nprobes: int, seed: int, dims=(32, 64, 128),
                     max_subset=64):
    """Uneven gallery subsets for batched search.

    Splits total_blocks into consecutive subsets of 1..max_subset blocks (seeded
    sizes), gives each subset a dimensionality from dims, and spreads nprobes
    probes over the subsets (every subset gets at least one probe while probes
    remain).  Returns (subsets, probe_subset): subsets is a list of
    (first_block, nblocks, d); probe_subset[i] is the subset probe i searches.
    """
    rng = np.random.default_rng([seed, 0x62617463])
    subsets = []
    b = 0
    while b < total_blocks:
        size = int(min(rng.integers(1, max_subset + 1), total_blocks - b))
        subsets.append((b, size, int(rng.choice(dims))))
        b += size
    order = list(range(len(subsets)))
    probe_subset = []
    for i in range(nprobes):
        if i < len(order):
            probe_subset.append(order[i])
        else:
            probe_subset.append(int(rng.integers(0, len(subsets))))
    return subsets, np.array(probe_subset, dtype=np.int64)
