"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

Each workload is decoded exactly as `bench.py --workload <name>` decodes it: the same seeded
frames (inputs.make_frames_chunked, seed 100), the same handle (perm_seed 1) and the library's
default launch shape. On every frame, properties that hold at any size are checked: the
returned information bits re-encode to the returned codeword, and the returned path metric is
that codeword's discrepancy with the LLRs (exactly, for integer LLRs). On a sample of frames
spread over the batch (the first and last CTA waves and random frames between), the decoded
words and metrics are compared with the oracle on the same inputs and the same permutation
table (from the independent Python sampler): bit-exact for integer LLRs, within the FP32
tolerance of tests/test_gpu_parity.py otherwise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402

PM_RTOL = 1e-4
MISMATCH_MAX = 0.01

# (bench workload, m, r, P, L, Eb/N0, frames per step, LLR type) as bench.py runs them
FULL = [
    ("rm29_p20_l4", 9, 2, 20, 4, 2.25, 1 << 18, "f32"),
    ("rm27_p8_l4", 7, 2, 8, 4, 3.0, 1 << 20, "i8"),
    ("rm25_p4_l2", 5, 2, 4, 2, 3.0, 1 << 21, "f32"),
    ("rm39_p16_l8", 9, 3, 16, 8, 4.0, 1 << 16, "f16"),
]


def _sample(nf, n_edge=64, n_mid=384, seed=0):
    rng = np.random.default_rng(seed)
    mid = rng.choice(np.arange(n_edge, nf - n_edge), size=n_mid, replace=False)
    return np.unique(np.concatenate([np.arange(n_edge), nf - n_edge + np.arange(n_edge), mid]))


@pytest.mark.parametrize("name,m,r,P,L,eb,nf,dt", FULL, ids=[f[0] for f in FULL])
def test_full_size_batch(name, m, r, P, L, eb, nf, dt):
    llr32, _ = I.make_frames_chunked(m, r, nf, eb, seed=100)
    if dt == "i8":
        x_np = I.quantize_i8(llr32)
    elif dt == "f16":
        x_np = I.to_f16(llr32)
    else:
        x_np = llr32
    del llr32
    dec = pkg.Decoder(m, r, P, L, perm_seed=1, dtype=dt)
    x = torch.from_numpy(x_np).cuda()
    bits, cw_w, pm_t, best_t = dec.decode_debug(x)
    torch.cuda.synchronize()
    w, c = dec.get_tuning()
    assert w >= 1 and c >= 1
    bits, cw_w, pm, best = bits.cpu().numpy(), cw_w.cpu().numpy(), pm_t.cpu().numpy().astype(np.float64), best_t.cpu().numpy()
    del x

    # every frame: a codeword with its own message, metric = its discrepancy
    worst = 0.0
    for c0 in range(0, nf, 1 << 16):
        c1 = min(nf, c0 + (1 << 16))
        info_c = pkg.unpack_bits(bits[c0:c1], dec.k)
        cw_c = pkg.unpack_bits(cw_w[c0:c1], dec.n)
        assert np.array_equal(I.encode(info_c, m, r), cw_c), c0
        y = x_np[c0:c1].astype(np.float64)
        disc = np.sum(np.abs(y) * (cw_c != (y < 0)), axis=1)
        if dt == "i8":
            assert np.array_equal(pm[c0:c1], disc), c0
        else:
            tol = PM_RTOL * (np.abs(disc) + np.abs(y).mean(axis=1))
            worst = max(worst, float(np.max(np.abs(pm[c0:c1] - disc) / tol)))
    assert worst <= 1.0, worst

    # sampled frames against the oracle, same table as the handle's seed
    idx = _sample(nf)
    perms = I.perm_table(m, r, P, L, seed=1)
    assert np.array_equal(dec.get_perms().reshape(perms.shape), perms)
    y = x_np[idx]
    ref = O.decode(m, r, P, L, perms, y.astype(np.int64 if dt == "i8" else np.float64), integer=(dt == "i8"))
    cw = pkg.unpack_bits(cw_w[idx], dec.n)
    if dt == "i8":
        assert np.array_equal(cw, ref["cw"])
        assert np.array_equal(pkg.unpack_bits(bits[idx], dec.k), ref["info"])
        assert np.array_equal(pm[idx].astype(np.int64), ref["pm"])
        assert np.array_equal(best[idx], ref["best"])
    else:
        same = np.all(cw == ref["cw"], axis=1)
        assert 1.0 - same.mean() <= MISMATCH_MAX
        assert np.all(ref["margin"][~same] < PM_RTOL)
        s = np.abs(y.astype(np.float64)).mean(axis=1)
        d = np.abs(pm[idx][same] - ref["pm"][same])
        assert np.all(d <= PM_RTOL * (np.abs(ref["pm"][same]) + s[same]))
