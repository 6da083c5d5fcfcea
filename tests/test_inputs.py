"""Checks of the seeded input generator: Philox known answers, GA(m) sampling, the
Reed-Muller encoder and the channel/quantiser conventions."""
import os

import numpy as np
import pytest

from paper_2108_12550_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gm(m):
    g = np.array([[1, 0], [1, 1]], dtype=np.int64)
    out = np.array([[1]], dtype=np.int64)
    for _ in range(m):
        out = np.kron(out, g)
    return out


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        ctr = np.array([v[0:4]], dtype=np.uint32)
        out = I.philox4x32_10(ctr, (v[4], v[5]))[0]
        assert [int(t) for t in out] == v[6:10]


def test_info_set_size_and_rows():
    for m, r in [(3, 1), (5, 2), (7, 2), (9, 2), (9, 3)]:
        n, k = I.rm_dims(m, r)
        idx = I.info_set(m, r)
        assert len(idx) == k
        # information rows are those of weight >= d = 2^(m-r) (Section II-A)
        w = _gm(m).sum(axis=1)
        assert set(idx.tolist()) == set(np.nonzero(w >= 2 ** (m - r))[0].tolist())
    assert I.info_set(3, 1).tolist() == [3, 5, 6, 7]  # the paper's RM(1,3) example


def test_encoder_matches_kronecker_matrix():
    rng = np.random.default_rng(0)
    for m, r in [(4, 2), (5, 2), (7, 3)]:
        n, k = I.rm_dims(m, r)
        u = rng.integers(0, 2, (20, k), dtype=np.uint8)
        full = np.zeros((20, n), dtype=np.int64)
        full[:, I.info_set(m, r)] = u
        assert np.array_equal(I.encode(u, m, r), (full @ _gm(m)) % 2)


def test_kronecker_power_is_the_subset_matrix_and_an_involution():
    """G^{(x)m} with G = [[1, 0], [1, 1]] has entry (i, j) = [j subset of i] (bits), and it is its
    own inverse over GF(2): the encoder x = u G^{(x)m} and the decoders' u = x G^{(x)m} invert
    each other."""
    for m in range(1, 10):
        g = _gm(m)
        i, j = np.meshgrid(np.arange(1 << m), np.arange(1 << m), indexing="ij")
        assert np.array_equal(g, ((i & j) == j).astype(g.dtype))
        assert np.array_equal((g.astype(np.int64) @ g) % 2, np.eye(1 << m, dtype=np.int64))


def test_rm25_minimum_distance_by_enumeration():
    m, r = 5, 2
    n, k = I.rm_dims(m, r)
    u = ((np.arange(1 << k)[:, None] >> np.arange(k)) & 1).astype(np.uint8)
    w = I.encode(u, m, r).sum(axis=1)
    assert w[0] == 0 and w[1:].min() == 2 ** (m - r)


def _apply(rec, s):
    idx = np.arange(1 << s)
    out = np.full(1 << s, int(rec[I.MAXM]), dtype=np.int64)
    for t in range(s):
        out ^= np.where((idx >> t) & 1, int(rec[t]), 0)
    return out


def _frozen_zero(x, m, r):
    u = x.astype(np.int64) @ _gm(m) % 2  # G^{(x)m} is an involution over GF(2)
    frozen = np.setdiff1d(np.arange(1 << m), I.info_set(m, r))
    return np.all(u[:, frozen] == 0)


def test_ga_permutations_are_automorphisms():
    rng = np.random.default_rng(1)
    for m, r in [(5, 2), (7, 2), (9, 3)]:
        tab = I.perm_table(m, r, 3, 2, seed=123)
        n, k = I.rm_dims(m, r)
        x = I.encode(rng.integers(0, 2, (16, k), dtype=np.uint8), m, r)
        for p in range(tab.shape[0]):
            for q in range(tab.shape[1]):
                s = m if q < 2 else m - (q - 2) // 4
                pi = _apply(tab[p, q], s)
                assert sorted(pi.tolist()) == list(range(1 << s))  # a bijection
                if s == m:
                    assert _frozen_zero(x[:, pi], m, r)  # maps codewords to codewords
                else:
                    # deeper levels act on the node RM(r - (m - s), s)
                    rs = r - (m - s)
                    _, ks = I.rm_dims(s, rs)
                    xs = I.encode(rng.integers(0, 2, (8, ks), dtype=np.uint8), s, rs)
                    assert _frozen_zero(xs[:, pi], s, rs)


def test_perm_table_layout_and_determinism():
    a = I.perm_table(9, 3, 2, 4, seed=77)
    b = I.perm_table(9, 3, 2, 4, seed=77)
    c = I.perm_table(9, 3, 2, 4, seed=78)
    assert a.shape == (2, 4 + 2 * 8, 11)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a[:, :12, 9] == 0) and np.all(a[:, 12:, 8:10] == 0)  # unused columns


def test_channel_and_quantisers():
    s2 = I.sigma2_for(2.0, 9, 2)
    assert abs(s2 - 1.0 / (2 * 46 / 512 * 10 ** 0.2)) < 1e-15
    fr = I.make_frames(5, 2, 2000, 3.0, seed=4)
    z = fr["llr"] * fr["sigma2"] / 2 - (1 - 2.0 * fr["x"])
    assert abs(z.var() - fr["sigma2"]) < 0.05 * fr["sigma2"]
    q = I.quantize_i8(np.array([0.125, 0.375, -0.125, 100.0, -100.0, 0.3]))
    assert q.tolist() == [0, 2, 0, 127, -127, 1]  # half to even, saturate at +-127
    nl = I.noiseless_frames(5, 2, 4, seed=1)
    assert np.all((nl["llr"] < 0) == (nl["x"] == 1))


def test_torch_frame_generator_encodes_like_numpy():
    torch = pytest.importorskip("torch")
    g = torch.Generator()
    g.manual_seed(3)
    for m, r in [(5, 2), (9, 3)]:
        u, llr = I.make_frames_torch(m, r, 50, 40.0, g, device="cpu")  # 40 dB: signs are the codeword
        x = I.encode(u.numpy(), m, r)
        assert np.array_equal((llr.numpy() < 0).astype(np.uint8), x)
        assert llr.dtype == torch.float32
