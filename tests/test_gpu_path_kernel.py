"""The path-per-thread kernel (one thread per list path, two for m = 8; RM(2, m) with
4 <= m <= 8 and RM(3, m) with 5 <= m <= 7, L <= 8)
against the warp-per-decoder kernel and the oracle, through the C ABI.

Both kernels run the same method (Algorithms 2-5), so on integer LLRs (INT8, INT16, FP32
holding integers) every output is identical: information bits, codewords, metrics, winning
decoder. On real-valued FP32 and FP16 LLRs they may differ only where two FHTL candidates of
one path round to the same FP32 metric; the bound below is far above the measured rate, and
every returned metric must be the discrepancy of the returned word."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402


def _run(dec, x):
    bits, cw, pm, best = dec.decode_debug(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return (bits.cpu().numpy(), cw.cpu().numpy(), pm.cpu().numpy(), best.cpu().numpy())


def _both(m, r, P, L, x, dtype, perms):
    out = {}
    for k in ("warp", "path"):
        dec = pkg.Decoder(m, r, P, L, dtype=dtype, perms=perms)
        dec.set_kernel(k)
        out[k] = _run(dec, x)
    return out["warp"], out["path"]


# (m, P, L, frames): every list size, batches of decoders (P * L > 32), idle decoder slots
# (P * L not a power of two) and ragged frame counts (not a multiple of the frames per warp)
CASES = [(m, r, P, L, nf) for (m, r) in [(4, 2), (5, 2), (6, 2), (7, 2), (8, 2), (5, 3), (6, 3), (7, 3)]
         for (P, L, nf) in [(1, 1, 333), (3, 2, 250), (8, 4, 200), (20, 4, 61), (2, 8, 97), (5, 8, 33)]]


@pytest.mark.parametrize("m,r,P,L,nf", CASES, ids=lambda v: str(v))
def test_integer_llrs_identical_to_the_warp_kernel(m, r, P, L, nf):
    fr = I.make_frames(m, r, nf, 1.5 + 0.25 * L, seed=500 + 10 * m + L)
    q = I.quantize_i8(fr["llr"])
    perms = I.perm_table(m, r, P, L, seed=m + 3 * L + P)
    w, p = _both(m, r, P, L, q, "i8", perms)
    for a, b, name in zip(w, p, ("bits", "cw", "pm", "best")):
        assert np.array_equal(a, b), name


@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (7, 2, 8, 4), (6, 2, 3, 8), (4, 2, 2, 1), (8, 2, 8, 4),
                                     (8, 2, 3, 8), (8, 2, 2, 1), (5, 3, 3, 4), (6, 3, 2, 8), (7, 3, 8, 4), (7, 3, 1, 1)])
def test_integer_llrs_match_the_oracle(m, r, P, L):
    fr = I.make_frames(m, r, 300, 2.0, seed=70 + m)
    q = I.quantize_i8(fr["llr"])
    perms = I.perm_table(m, r, P, L, seed=9 * m + L)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    dec.set_kernel("path")
    bits, cw, pm, best = _run(dec, q)
    assert np.array_equal(pkg.unpack_bits(cw, dec.n), ref["cw"])
    assert np.array_equal(pm.astype(np.int64), ref["pm"]) and np.array_equal(best, ref["best"])
    assert np.array_equal(pkg.unpack_bits(bits, dec.k), ref["info"])


@pytest.mark.parametrize("dtype", ["f32", "f16", "i16"])
@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (7, 2, 8, 4), (6, 2, 20, 8), (8, 2, 20, 4), (7, 3, 8, 4)])
def test_other_input_types_agree_with_the_warp_kernel(m, r, P, L, dtype):
    fr = I.make_frames(m, r, 1500, 2.5, seed=90 + m + L)
    if dtype == "f32":
        x = fr["llr"].astype(np.float32)
    elif dtype == "f16":
        x = fr["llr"].astype(np.float16)
    else:
        x = np.clip(np.rint(fr["llr"] * 256), -32767, 32767).astype(np.int16)
    perms = I.perm_table(m, r, P, L, seed=5 * m + L)
    w, p = _both(m, r, P, L, x, dtype, perms)
    if dtype == "i16":
        for a, b in zip(w, p):
            assert np.array_equal(a, b)
        return
    same = np.all(w[1] == p[1], axis=1)
    assert same.mean() >= 0.998, same.mean()
    # every returned metric is the discrepancy of the returned word
    xf = x.astype(np.float64)
    cw = pkg.unpack_bits(p[1], 1 << m)
    disc = np.sum(np.abs(xf) * (cw != (xf < 0)), axis=1)
    np.testing.assert_allclose(p[2], disc, rtol=1e-4, atol=1e-4 * np.abs(xf).mean())


def test_tuning_shapes_and_tiny_batches():
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 700, 2.0, seed=12)
    q = I.quantize_i8(fr["llr"])
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perm_seed=4)
    dec.set_kernel("path")
    ref = _run(dec, q)
    for w in (1, 2, 3, 4):
        dec.set_tuning(w, 0)
        assert all(np.array_equal(a, b) for a, b in zip(ref, _run(dec, q))), w
    dec.set_tuning(0, 1)
    assert all(np.array_equal(a, b) for a, b in zip(ref, _run(dec, q)))
    dec.set_tuning(0, 0)
    for n in (1, 2, 5):  # fewer frames than a warp decodes at once
        got = _run(dec, q[:n])
        assert all(np.array_equal(a[:n], b) for a, b in zip(ref, got)), n
    small = pkg.Decoder(5, 2, 1, 1, dtype="i8", perm_seed=2)  # 32 frames per warp
    small.set_kernel("path")
    fr5 = I.make_frames(5, 2, 77, 2.0, seed=3)
    q5 = I.quantize_i8(fr5["llr"])
    a = _run(small, q5)
    small.set_kernel("warp")
    assert all(np.array_equal(x, y) for x, y in zip(a, _run(small, q5)))


def test_decoder_batches_split_over_the_warps_of_a_cta():
    # RM(2,8) P=20 L=4: five batches of four decoders per frame; one to four warps per CTA
    # split them, and the warps' best decoders meet in shared memory
    m, r, P, L = 8, 2, 20, 4
    fr = I.make_frames(m, r, 203, 2.0, seed=15)
    q = I.quantize_i8(fr["llr"])
    perms = I.perm_table(m, r, P, L, seed=16)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    dec.set_kernel("path")
    for w in (1, 2, 3, 4):
        dec.set_tuning(w, 0)
        bits, cw, pm, best = _run(dec, q)
        assert np.array_equal(pkg.unpack_bits(cw, dec.n), ref["cw"]), w
        assert np.array_equal(best, ref["best"]) and np.array_equal(pm.astype(np.int64), ref["pm"]), w


def test_auto_takes_each_kernel_by_launch_size():
    # 'auto' gives small launches to the warp kernel and large ones to the path kernel; on
    # integer LLRs both decode identically, so the results of one batch decoded whole and in
    # small pieces agree
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 5000, 2.0, seed=14)
    q = I.quantize_i8(fr["llr"])
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perm_seed=4)
    whole = _run(dec, q)  # >= 2,048 frames: path-per-thread kernel
    parts = [_run(dec, q[i:i + 500]) for i in range(0, 5000, 500)]  # warp kernel
    for k in range(4):
        assert np.array_equal(whole[k], np.concatenate([p[k] for p in parts])), k


def test_kernel_choice_is_validated():
    with pytest.raises(pkg.RmdecError):
        pkg.Decoder(9, 2, 4, 4).set_kernel("path")  # no path-per-thread kernel for m = 9
    pkg.Decoder(8, 2, 20, 8).set_kernel("path")
    with pytest.raises(pkg.RmdecError):
        pkg.Decoder(8, 3, 4, 4).set_kernel("path")  # nor for RM(3, 8)
    pkg.Decoder(6, 3, 4, 4).set_kernel("path")
    with pytest.raises(pkg.RmdecError):
        pkg.Decoder(6, 2, 4, 16).set_kernel("path")  # nor for L = 16
    pkg.Decoder(7, 2, 20, 8).set_kernel("path")


@pytest.mark.parametrize("m,r,P,L,path", [
    (7, 2, 8, 4, True), (5, 2, 128, 4, True), (6, 3, 16, 8, True), (8, 2, 20, 4, True), (7, 3, 1, 4, True),
    (6, 2, 32, 8, True), (7, 2, 1, 1, False), (8, 2, 8, 8, False), (5, 2, 64, 8, False), (6, 3, 20, 8, False),
    (8, 2, 32, 4, False), (7, 3, 8, 8, False), (7, 2, 2, 4, False), (9, 2, 20, 4, False)])
def test_auto_takes_the_path_kernel_only_where_it_was_measured_faster(m, r, P, L, path):
    # large launches go to the path-per-thread kernel only for the P and L where it decoded
    # faster than the warp kernel (large P leaves it few CTAs per SM; L = 8 costs it more)
    dec = pkg.Decoder(m, r, P, L, perm_seed=1)
    assert dec.kernel_for(1 << 16) == ("path" if path else "warp")
    assert dec.kernel_for(64) == "warp"
    if (m, r) != (9, 2):
        fresh = pkg.Decoder(m, r, P, L, perm_seed=1)
        fresh.set_kernel("warp")
        dec.set_kernel("path")  # forced, it takes every launch
        assert dec.kernel_for(1) == "path"
        dec.set_kernel("warp")  # and back: the warp kernel in its own launch shape
        assert dec.kernel_for(1 << 16) == "warp"
        assert dec.get_tuning() == fresh.get_tuning()


@pytest.mark.parametrize("kernel", ["path", "warp"])
@pytest.mark.parametrize("m,r,P,L", [(8, 2, 8, 4), (8, 2, 3, 8), (7, 2, 8, 4), (6, 2, 4, 2), (7, 3, 4, 4), (6, 3, 2, 8),
                                     (9, 2, 20, 4), (9, 3, 4, 8)])
def test_full_range_int8_codes_match_the_oracle(m, r, P, L, kernel):
    # INT8 codes over their whole range, -128 included (the quantiser stops at -127): frames
    # all -128 or all 127 reach the largest spectrum values, 2^m x 128, where the path kernel's
    # packed candidate keys have the fewest spare bits; all-zero frames tie everything
    if kernel == "path" and m == 9:
        pytest.skip("no path-per-thread kernel for length 512")
    n = 1 << m
    rng = np.random.default_rng(1000 + 10 * m + L)
    q = rng.integers(-128, 128, size=(96, n)).astype(np.int8)
    q[0], q[1], q[3] = -128, 127, 0
    q[2] = np.where(np.arange(n) % 3 == 0, -128, 127)
    fr = I.make_frames(m, r, 40, 2.0, seed=20 + m)
    q[4:44] = np.clip(np.rint(fr["llr"] * 16), -128, 127).astype(np.int8)  # saturated channel frames
    perms = I.perm_table(m, r, P, L, seed=7 * m + L)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    dec.set_kernel(kernel)
    bits, cw, pm, best = _run(dec, q)
    assert np.array_equal(pkg.unpack_bits(cw, dec.n), ref["cw"])
    assert np.array_equal(pm.astype(np.int64), ref["pm"]) and np.array_equal(best, ref["best"])
    assert np.array_equal(pkg.unpack_bits(bits, dec.k), ref["info"])
