"""Seeded synthetic inputs shared by the CPU oracle, the GPU decoder's tests and the benchmark.

This module holds no decoding arithmetic. It produces what a transmitter and a channel
produce, plus the random draws the decoder consumes:

* the Reed-Muller code's information set and an encoder x = u G^{(x)m} (Section II-A),
  used only to make transmitted codewords;
* BPSK over AWGN and the channel LLR 2y/sigma^2 (Section II-A);
* the INT8 and FP16 quantisers of the LLRs;
* the table of affine permutations x -> Ax + b drawn from GA(m) (Algorithm 2: the
  initial permutations pi^init_l and the 2L candidate permutations per permuted node).

The permutation table is drawn with Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11) written here from that paper's definition.
The GPU library carries its own independent implementation of the same generator, so a
handle built from a seed can be checked against this module without either side reading
the other's code.

Permutation record layout (shared by every consumer): 11 uint16 per element of GA(s),
``[c_0, ..., c_9, b]`` where ``c_t = A e_t`` is column t of A (only ``t < s`` used) and the
element maps index i to ``b XOR (XOR over set bits t of i of c_t)``.
Per decoder p the table holds ``L`` initial permutations of GA(m), then for each permuted
level j = 0 .. r-2 (the node RM(r-j, m-j)) ``2L`` candidates of GA(m-j).
"""
from __future__ import annotations

import math

import numpy as np

MAXM = 10
PERM_REC = MAXM + 1  # uint16 entries per permutation record

# Philox4x32 round multipliers and Weyl key increments (SC'11, Section 4).
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

PERM_DOMAIN_TAG = 0x5045524D  # 'PERM' in the last counter word of permutation draws


def philox4x32_10(counters: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds on an (N, 4) uint32 counter array, returns (N, 4) uint32."""
    c = np.asarray(counters, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0 = np.uint64(key[0] & 0xFFFFFFFF)
    k1 = np.uint64(key[1] & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _PHILOX_W0) & _MASK32
            k1 = (k1 + _PHILOX_W1) & _MASK32
        p0 = c0 * _PHILOX_M0
        p1 = c2 * _PHILOX_M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


# --------------------------------------------------------------------------- code ---

def rm_dims(m: int, r: int) -> tuple[int, int]:
    """Length N = 2^m and dimension K = sum_{i<=r} C(m, i) of RM(r, m) (Section II-A)."""
    return 1 << m, sum(math.comb(m, i) for i in range(r + 1))


def info_set(m: int, r: int) -> np.ndarray:
    """Information set I = {i : w_i >= d}: row i of G^{(x)m} has weight 2^popcount(i) and
    d = 2^(m-r), so I = {i : popcount(i) >= m - r}, ascending (Section II-A)."""
    n = 1 << m
    idx = np.arange(n)
    pc = np.array([bin(i).count("1") for i in idx])
    return idx[pc >= m - r]


def encode(u_info: np.ndarray, m: int, r: int) -> np.ndarray:
    """x = u G^{(x)m} over GF(2) with u zero on the frozen set (Section II-A).

    u_info: (F, K) uint8 message bits placed on I in ascending order. Returns (F, N) uint8.
    G = [[1,0],[1,1]], so G^{(x)m}[i][j] = 1 iff j is a bit-subset of i and
    x_j = XOR of u_i over i containing j: an in-place butterfly over the m index bits.
    """
    n = 1 << m
    u_info = np.asarray(u_info, dtype=np.uint8)
    x = np.zeros((u_info.shape[0], n), dtype=np.uint8)
    x[:, info_set(m, r)] = u_info
    for t in range(m):
        h = 1 << t
        x = x.reshape(-1, n // (2 * h), 2, h)
        x[:, :, 0, :] ^= x[:, :, 1, :]
        x = x.reshape(-1, n)
    return x


# ------------------------------------------------------------------------ channel ---

def sigma2_for(ebn0_db: float, m: int, r: int) -> float:
    """Noise variance for unit-energy BPSK at Eb/N0 with rate R = K/N: 1/(2 R 10^(Eb/N0/10))."""
    n, k = rm_dims(m, r)
    return 1.0 / (2.0 * (k / n) * 10.0 ** (ebn0_db / 10.0))


def make_frames(m: int, r: int, n_frames: int, ebn0_db: float, seed: int):
    """Random messages, codewords and FP64 channel LLRs alpha_m = 2y/sigma^2 with
    y = (1 - 2x) + z, z ~ N(0, sigma^2) (Section II-A).

    Returns dict with u (F,K) uint8, x (F,N) uint8, llr (F,N) float64, sigma2.
    """
    n, k = rm_dims(m, r)
    rng = np.random.Generator(np.random.Philox(key=seed))
    u = rng.integers(0, 2, size=(n_frames, k), dtype=np.uint8)
    x = encode(u, m, r)
    s2 = sigma2_for(ebn0_db, m, r)
    y = (1.0 - 2.0 * x) + rng.normal(0.0, math.sqrt(s2), size=(n_frames, n))
    return {"u": u, "x": x, "llr": 2.0 * y / s2, "sigma2": s2}


def noiseless_frames(m: int, r: int, n_frames: int, seed: int, amplitude: float = 4.0):
    """Frames whose LLR signs equal the transmitted BPSK symbols, with random magnitudes
    in [amplitude/2, amplitude] so that no two positions tie."""
    n, k = rm_dims(m, r)
    rng = np.random.Generator(np.random.Philox(key=seed))
    u = rng.integers(0, 2, size=(n_frames, k), dtype=np.uint8)
    x = encode(u, m, r)
    mag = rng.uniform(amplitude / 2, amplitude, size=(n_frames, n))
    return {"u": u, "x": x, "llr": (1.0 - 2.0 * x) * mag}


def quantize_i8(llr: np.ndarray, step: float = 0.25) -> np.ndarray:
    """INT8 LLR: round-half-to-even of llr/step, saturated to [-127, 127]."""
    return np.clip(np.rint(np.asarray(llr, dtype=np.float64) / step), -127, 127).astype(np.int8)


def to_f16(llr: np.ndarray) -> np.ndarray:
    return np.asarray(llr, dtype=np.float64).astype(np.float16)


# ------------------------------------------------------------------- permutations ---

def _bits_of_block(words: np.ndarray, nbits: int) -> np.ndarray:
    """Little-endian bit expansion of one 4x32-bit Philox block."""
    out = np.zeros(nbits, dtype=np.uint8)
    for q in range(nbits):
        out[q] = (int(words[q >> 5]) >> (q & 31)) & 1
    return out


def _gf2_rank(cols: list[int], s: int) -> int:
    rows = list(cols)
    rank = 0
    for bit in range(s):
        piv = next((i for i in range(rank, len(rows)) if (rows[i] >> bit) & 1), None)
        if piv is None:
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for i in range(len(rows)):
            if i != rank and (rows[i] >> bit) & 1:
                rows[i] ^= rows[rank]
        rank += 1
    return rank


def sample_ga(s: int, seed: int, p: int, q: int) -> np.ndarray:
    """One element of GA(s): A uniform in GL(s, 2) by rejection, b uniform in F_2^s.

    Draw `a` uses Philox counter (p, q, a, 'PERM') under key (seed_lo, seed_hi): bits
    [t*s, (t+1)*s) form column t of A and bits [s*s, s*s + s) form b. Draws repeat with
    a = 0, 1, ... until A is invertible. Returns an 11-entry uint16 record.
    """
    assert 1 <= s <= MAXM and s * s + s <= 128
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = 0
    while True:
        blk = philox4x32_10(np.array([[p, q, a, PERM_DOMAIN_TAG]], dtype=np.uint32), key)[0]
        bits = _bits_of_block(blk, s * s + s)
        cols = [int(sum(int(bits[t * s + i]) << i for i in range(s))) for t in range(s)]
        if _gf2_rank(cols, s) == s:
            rec = np.zeros(PERM_REC, dtype=np.uint16)
            rec[:s] = cols
            rec[MAXM] = sum(int(bits[s * s + i]) << i for i in range(s))
            return rec
        a += 1


def n_perm_levels(m: int, r: int) -> int:
    """Permuted nodes are the left spine RM(r, m), RM(r-1, m-1), ..., RM(2, m-r+2): the nodes
    with 1 < r_v < m_v - 1 visited before the first order-1 node (Algorithm 2)."""
    return max(0, r - 1) if 1 < r < m - 1 else 0


def perms_per_decoder(m: int, r: int, L: int) -> int:
    return L + n_perm_levels(m, r) * 2 * L


def perm_table(m: int, r: int, P: int, L: int, seed: int) -> np.ndarray:
    """(P, L + (r-1)*2L, 11) uint16 table; see the module docstring for the layout."""
    nq = perms_per_decoder(m, r, L)
    tab = np.zeros((P, nq, PERM_REC), dtype=np.uint16)
    for p in range(P):
        for q in range(nq):
            s = m if q < L else m - (q - L) // (2 * L)
            tab[p, q] = sample_ga(s, seed, p, q)
    return tab


def ga_record(cols, b: int = 0) -> np.ndarray:
    """GA record [c_0 .. c_9, b] from the columns of A (c_t = A e_t) and the shift b."""
    rec = np.zeros(PERM_REC, dtype=np.uint16)
    rec[:len(cols)] = cols
    rec[PERM_REC - 1] = b
    return rec


def selection_case(level: str, n_frames: int, seed: int, integer: bool = False):
    """Frames and permutation records whose candidate reliabilities are ordered by
    construction, for checks of the permutation selection with P = 1, L = 1.

    Three GA(5) candidates: A and A2 map the top index bit to a = 16, B to a = 1 (A2 also maps
    index bit 3 elsewhere than A, so the two split the next node differently). The frame
    magnitudes are small on S = {0, 16, 5, 21} (closed under xor 16, disjoint from S xor 1)
    and large elsewhere, so a left child pairing positions {j, j xor 16} meets the small
    values two at a time and one pairing {j, j xor 1} meets them one at a time. level "root":
    RM(2,5), the candidates act on the root; "deeper": RM(3,6) with identity root maps and a
    large right half, the candidates act on the node RM(2,5). Signs are uniform. integer=True
    gives integer magnitudes (1000-1160 and 1-3, right half 2000-2100). Returns
    dict(m, r, head (records before the two candidates), A, A2, B, llr (F, 2^m) float64).
    """
    rng = np.random.default_rng(seed)
    if level == "root":
        m, r = 5, 2
        head = [ga_record([1, 2, 4, 8, 16])]
    elif level == "deeper":
        m, r = 6, 3
        i6 = ga_record([1, 2, 4, 8, 16, 32])
        head = [i6, i6, i6]
    else:
        raise ValueError(level)
    n = 1 << m
    small = [0, 16, 5, 21]
    if integer:  # 14 x 1000 + 2 x 1 > 12 x 1160 + 4 x 3: the order holds for every draw
        mag = 1000.0 + rng.integers(0, 161, (n_frames, n))
        mag[:, small] = 1.0 + rng.integers(0, 3, (n_frames, len(small)))
        if level == "deeper":
            mag[:, 32:] = 2000.0 + rng.integers(0, 101, (n_frames, 32))
    else:
        mag = 1.0 + 0.1 * rng.random((n_frames, n))
        mag[:, small] = 0.01 * (1.0 + rng.random((n_frames, len(small))))
        if level == "deeper":
            mag[:, 32:] = 10.0 + rng.random((n_frames, 32))
    llr = np.where(rng.random((n_frames, n)) < 0.5, -1.0, 1.0) * mag
    return {"m": m, "r": r, "head": head, "A": ga_record([1, 2, 4, 8, 16]),
            "A2": ga_record([1, 2, 8, 4, 16], b=6), "B": ga_record([16, 2, 4, 8, 1]), "llr": llr}


SSC_STREAM = 0x53534300  # counter word 0 of the Aut-SSC permutation draws


def ssc_perm_table(m: int, P_ssc: int, seed: int) -> np.ndarray:
    """(P_ssc, 11) uint16 GA(m) records for the Aut-SSC-P baseline (counter word 0 = 'SSC\\0')."""
    return np.stack([sample_ga(m, seed, SSC_STREAM, q) for q in range(P_ssc)])


def make_frames_chunked(m: int, r: int, n_frames: int, ebn0_db: float, seed: int, chunk: int = 1 << 16):
    """Large batches of make_frames, generated in chunks of `chunk` frames, chunk c0 with seed
    seed * 1000003 + c0 (the full-size benchmark batches). Returns (llr float32 [F,N],
    u uint8 [F,K])."""
    n, k = rm_dims(m, r)
    llr = np.empty((n_frames, n), dtype=np.float32)
    u = np.empty((n_frames, k), dtype=np.uint8)
    for c0 in range(0, n_frames, chunk):
        c1 = min(n_frames, c0 + chunk)
        fr = make_frames(m, r, c1 - c0, ebn0_db, seed=seed * 1000003 + c0)
        llr[c0:c1] = fr["llr"]
        u[c0:c1] = fr["u"]
    return llr, u


def make_frames_torch(m: int, r: int, n_frames: int, ebn0_db: float, generator, device="cuda"):
    """The same transmitter and channel as make_frames, on a torch device (for sweeps whose
    frames are too many to stage from the host): uniform messages, x = u G^{(x)m}, BPSK over
    AWGN, FP32 LLRs 2y/sigma^2. Returns (u uint8 [F,K], llr float32 [F,N])."""
    import torch

    n, k = rm_dims(m, r)
    u = torch.randint(0, 2, (n_frames, k), dtype=torch.uint8, device=device, generator=generator)
    x = torch.zeros((n_frames, n), dtype=torch.uint8, device=device)
    x[:, torch.as_tensor(info_set(m, r), device=device)] = u
    for t in range(m):
        h = 1 << t
        v = x.view(n_frames, n // (2 * h), 2, h)
        v[:, :, 0, :] ^= v[:, :, 1, :]
    s2 = sigma2_for(ebn0_db, m, r)
    z = torch.randn((n_frames, n), dtype=torch.float32, device=device, generator=generator)
    y = (1.0 - 2.0 * x.float()) + math.sqrt(s2) * z
    return u, (2.0 / s2) * y
