"""GPU parity of the CUDA decoder (through the C ABI) against the CPU oracle.

Integer LLRs (I8, I16, and F32 holding integer values) must match the oracle's exact integer
mode bit for bit: information bits, codewords, path metrics and winning decoder. Real-valued
FP32/FP16 LLRs are compared with the FP64 oracle within the stated tolerance: identical
decoded words except at near-ties (rare), path metrics within 1e-4 relative, and on every
frame the GPU's metric equals the discrepancy of the word it returned.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402

PM_RTOL = 1e-4          # FP32 path metrics vs FP64 (relative, plus the frame's mean |LLR|)
MISMATCH_MAX = 0.01     # largest tolerated fraction of FP32 frames decided differently


def _gpu_decode(dec, llr_np):
    x = torch.from_numpy(np.ascontiguousarray(llr_np)).cuda()
    bits, cw, pm, best = dec.decode_debug(x)
    torch.cuda.synchronize()
    return (pkg.unpack_bits(bits.cpu().numpy(), dec.k), pkg.unpack_bits(cw.cpu().numpy(), dec.n),
            pm.cpu().numpy(), best.cpu().numpy())


def _disc(llr, cw):
    return np.sum(np.abs(llr) * (cw != (llr < 0)), axis=-1)


CONFIGS = [  # (m, r, P, L, Eb/N0, frames)
    (4, 2, 2, 8, 2.0, 600),
    (5, 2, 4, 2, 3.0, 3000),     # RM(2,5), P=4, L=2 (the small benchmark case)
    (5, 3, 3, 4, 4.0, 1000),     # the paper's Fig. 3 example code, two permuted levels
    (6, 2, 3, 1, 2.0, 1000),
    (6, 3, 2, 8, 4.0, 500),
    (7, 2, 8, 4, 2.0, 2000),     # RM(2,7), P=8, L=4
    (8, 2, 8, 4, 2.5, 600),
    (9, 2, 20, 4, 2.25, 333),    # RM(2,9), P=20, L=4 (ragged frame count)
    (9, 3, 16, 8, 4.0, 150),     # RM(3,9), P=16, L=8
    (10, 2, 3, 4, 2.0, 120),     # RM(2,10) (length 1024)
    (10, 2, 2, 8, 2.0, 60),
    (10, 3, 2, 2, 3.0, 90),      # RM(3,10), two permuted levels
    (10, 3, 1, 8, 3.0, 40),
    (5, 2, 3, 16, 1.5, 300),     # L = 16: the paper's Fig. 4 and 5 list sizes beyond 8
    (7, 3, 2, 16, 2.5, 120),
    (9, 2, 2, 16, 1.5, 80),
    (9, 3, 1, 16, 2.5, 40),
    (10, 2, 1, 16, 1.5, 16),
    (6, 4, 3, 2, 2.0, 400),      # RM(4, m): three permuted levels (the paper's Fig. 4 and 5 codes)
    (7, 4, 2, 16, 3.0, 100),
    (8, 4, 4, 4, 3.0, 200),
    (9, 4, 2, 8, 3.5, 60),
    (4, 2, 2, 32, 1.5, 200),     # L = 32 (64 candidates per permuted node and SPC split)
    (6, 3, 2, 32, 2.0, 100),
    (8, 2, 1, 32, 1.5, 40),
    (9, 4, 1, 32, 3.0, 12),
]


@pytest.mark.parametrize("m,r,P,L,eb,nf", CONFIGS, ids=lambda v: str(v))
def test_integer_llrs_bit_exact(m, r, P, L, eb, nf):
    fr = I.make_frames(m, r, nf, eb, seed=100 + m * 10 + r)
    perms = I.perm_table(m, r, P, L, seed=m * 7 + L)
    q = I.quantize_i8(fr["llr"])
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"])
    assert np.array_equal(info, ref["info"])
    assert np.array_equal(pm.astype(np.int64), ref["pm"])
    assert np.array_equal(best, ref["best"])
    # the same kernel on FP32 inputs holding the integer codes is exact too
    dec.set_dtype("f32")
    info2, cw2, pm2, best2 = _gpu_decode(dec, q.astype(np.float32))
    assert np.array_equal(cw2, ref["cw"]) and np.array_equal(pm2.astype(np.int64), ref["pm"])
    assert np.array_equal(best2, ref["best"])


@pytest.mark.parametrize("level", ["root", "deeper"])
def test_constructed_permutation_selection_bit_exact(level):
    """The oracle's selection pins on the GPU, which sums LM over the pairs {j, j xor a}
    instead of gathering each candidate: the larger LM wins in either order, and on equal LM
    the earlier candidate wins. Integer-valued LLRs (FP32), bit-exact against the oracle."""
    c = I.selection_case(level, 700, seed=5, integer=True)
    m, r = c["m"], c["r"]
    y = c["llr"].astype(np.int64)
    for c0, c1 in (("A", "B"), ("B", "A"), ("A", "A2"), ("A2", "A"), ("B", "B")):
        tab = np.stack(c["head"] + [c[c0], c[c1]])[None]
        ref = O.decode(m, r, 1, 1, tab, y, integer=True, want_margin=False)
        dec = pkg.Decoder(m, r, 1, 1, dtype="f32", perms=tab)
        info, cw, pm, best = _gpu_decode(dec, y.astype(np.float32))
        assert np.array_equal(cw, ref["cw"]), (c0, c1)
        assert np.array_equal(pm.astype(np.int64), ref["pm"]), (c0, c1)
        assert np.array_equal(info, ref["info"]), (c0, c1)


def test_tied_decoders_resolve_to_the_earliest_under_every_shape():
    """Decoder 2 repeats decoder 0's table, so the two tie exactly on every frame; the winner
    over decoders (Algorithm 5, strict <) must be the oracle's, never decoder 2, whether the two
    run in different warps of a CTA or one after the other in the same warp."""
    m, r, P, L = 7, 2, 4, 2
    tab = I.perm_table(m, r, P, L, seed=23)
    tab[2] = tab[0]
    fr = I.make_frames(m, r, 800, 1.5, seed=41)
    q = I.quantize_i8(fr["llr"])
    ref = O.decode(m, r, P, L, tab, q.astype(np.int64), integer=True, want_margin=False)
    assert len(set(ref["best"].tolist())) >= 3 and not np.any(ref["best"] == 2)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=tab)
    for w in (1, 2, 3, 4):
        dec.set_tuning(w, 0)
        info, cw, pm, best = _gpu_decode(dec, q)
        assert np.array_equal(best, ref["best"]), w
        assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["pm"]), w


@pytest.mark.parametrize("m,r,P,L", [(7, 2, 8, 4), (9, 2, 4, 4)])
def test_i16_llrs_bit_exact(m, r, P, L):
    fr = I.make_frames(m, r, 400, 2.0, seed=5)
    q = np.clip(np.rint(fr["llr"] * 256), -32767, 32767).astype(np.int16)  # step 2^-8
    perms = I.perm_table(m, r, P, L, seed=3)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i16", perms=perms)
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["pm"])
    assert np.array_equal(best, ref["best"])


def _fp_compare(m, r, P, L, llr64, gpu_llr, dtype):
    perms = I.perm_table(m, r, P, L, seed=11)
    ref = O.decode(m, r, P, L, perms, llr64)
    dec = pkg.Decoder(m, r, P, L, dtype=dtype, perms=perms)
    info, cw, pm, best = _gpu_decode(dec, gpu_llr)
    scale = np.mean(np.abs(llr64), axis=1)
    # every returned metric is the discrepancy of the returned word
    np.testing.assert_allclose(pm, _disc(llr64, cw), rtol=PM_RTOL, atol=PM_RTOL * scale.max())
    same = np.all(cw == ref["cw"], axis=1)
    mismatch = 1.0 - same.mean()
    assert mismatch <= MISMATCH_MAX, mismatch
    d = np.abs(pm[same] - ref["pm"][same])
    assert np.all(d <= PM_RTOL * (np.abs(ref["pm"][same]) + scale[same])), d.max()
    # decisions differ only where the oracle saw a near-tie
    assert np.all(ref["margin"][~same] < PM_RTOL)
    return mismatch


@pytest.mark.parametrize("m,r,P,L,eb,nf", [(5, 2, 4, 2, 3.0, 3000), (7, 2, 8, 4, 2.0, 2000),
                                          (9, 2, 20, 4, 2.25, 400), (9, 3, 16, 8, 4.0, 150)],
                         ids=lambda v: str(v))
def test_fp32_within_tolerance(m, r, P, L, eb, nf):
    fr = I.make_frames(m, r, nf, eb, seed=77)
    _fp_compare(m, r, P, L, fr["llr"], fr["llr"].astype(np.float32), "f32")


def test_fp16_within_tolerance():
    m, r, P, L = 9, 3, 16, 8
    fr = I.make_frames(m, r, 150, 4.0, seed=78)
    h = I.to_f16(fr["llr"])
    _fp_compare(m, r, P, L, h.astype(np.float64), h, "f16")


@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (9, 2, 20, 4), (9, 3, 16, 8), (5, 3, 2, 1)])
def test_noiseless_frames_decode_exactly(m, r, P, L):
    nl = I.noiseless_frames(m, r, 64, seed=9)
    dec = pkg.Decoder(m, r, P, L, perm_seed=4)
    info, cw, pm, best = _gpu_decode(dec, nl["llr"].astype(np.float32))
    assert np.array_equal(info, nl["u"]) and np.all(np.abs(pm) <= 1e-5 * np.abs(nl["llr"]).sum(axis=1))


def test_library_seeded_tables_end_to_end():
    """A handle built from a seed (library sampler, root composition on the device side)
    decodes like the oracle given the independently generated table for the same seed."""
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 500, 1.5, seed=21)
    q = I.quantize_i8(fr["llr"])
    dec = pkg.Decoder(m, r, P, L, perm_seed=2718, dtype="i8")
    ref = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=2718), q.astype(np.int64), integer=True)
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["pm"])


def test_edge_cases_empty_single_and_determinism():
    m, r, P, L = 9, 2, 20, 4
    dec = pkg.Decoder(m, r, P, L, perm_seed=1)
    empty = torch.empty((0, 512), dtype=torch.float32, device="cuda")
    out = dec.decode(empty)
    assert out.shape == (0, 2)
    fr = I.make_frames(m, r, 1, 2.0, seed=3)
    one = torch.from_numpy(fr["llr"].astype(np.float32)).cuda()
    a = dec.decode(one).cpu()
    b = dec.decode(one).cpu()
    assert torch.equal(a, b)
    # all-zero LLRs: every decision is a tie; output must be a valid, deterministic codeword
    z = torch.zeros((3, 512), dtype=torch.float32, device="cuda")
    bits, cw, pm, best = dec.decode_debug(z)
    assert torch.all(pm == 0)
    q = torch.zeros((3, 512), dtype=torch.int8, device="cuda")
    dec.set_dtype("i8")
    bits2, cw2, _, _ = dec.decode_debug(q)
    assert torch.equal(cw, cw2)
    ref = O.decode(m, r, P, L, dec.get_perms().reshape(P, -1, 11), np.zeros((3, 512), np.int64), integer=True)
    assert np.array_equal(pkg.unpack_bits(cw2.cpu().numpy(), 512), ref["cw"])
    # saturated LLRs (+-127 everywhere, the quantiser's maximum) also decode exactly
    sat = np.where(I.noiseless_frames(m, r, 8, seed=2)["llr"] < 0, -127, 127).astype(np.int8)
    ref = O.decode(m, r, P, L, dec.get_perms().reshape(P, -1, 11), sat.astype(np.int64), integer=True)
    info, cw3, pm3, _ = _gpu_decode(dec, sat)
    assert np.array_equal(cw3, ref["cw"]) and np.all(pm3 == 0)


def test_host_entry_point_and_tickets():
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 1000, 2.0, seed=31)
    x = fr["llr"].astype(np.float32)
    dec = pkg.Decoder(m, r, P, L, perm_seed=5)
    dev = dec.decode(torch.from_numpy(x).cuda()).cpu()
    host_in = torch.from_numpy(x).pin_memory()
    host_out = torch.empty((1000, dec.kw), dtype=torch.int32).pin_memory()
    dec.decode_host(host_in, host_out)
    assert torch.equal(dev, host_out)
    s = torch.cuda.Stream()
    xin = torch.from_numpy(x).cuda()
    out = torch.empty((1000, dec.kw), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        t = dec.submit(xin, out, stream=s)
    assert dec.poll(t, timeout_us=10_000_000) == pkg.OK
    assert torch.equal(out.cpu(), dev)
    with pytest.raises(pkg.RmdecError):
        dec.poll(t, 0)  # retired ticket


@pytest.mark.parametrize("m,r,Ps", [(7, 2, 32), (9, 2, 64), (6, 3, 16), (9, 2, 512)])
def test_aut_ssc_bit_exact(m, r, Ps):
    # (9, 2, 512) is the size of the paper's Aut-SSC-512 comparison on RM(2,9)
    fr = I.make_frames(m, r, 300 if Ps > 64 else 400, 2.0, seed=41)
    q = I.quantize_i8(fr["llr"])
    perms = I.ssc_perm_table(m, Ps, seed=6)
    ref = O.aut_ssc(m, r, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, Ps, algo="autssc", perms=perms, dtype="i8")
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["disc"])
    assert np.array_equal(best, ref["best"])


@pytest.mark.parametrize("m,r,L", [(9, 2, 4), (7, 2, 8), (9, 3, 8), (5, 2, 1)])
def test_fhtfscl_variant_bit_exact(m, r, L):
    fr = I.make_frames(m, r, 400, 2.5, seed=61)
    q = I.quantize_i8(fr["llr"])
    ref = O.decode_fhtfscl(m, r, L, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, 1, L, algo="fhtfscl", dtype="i8")
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["pm"])


def test_p100_l1_bit_exact():
    m, r, P, L = 9, 2, 100, 1  # the paper's p-FHT-FSCL-1-100
    fr = I.make_frames(m, r, 200, 1.5, seed=62)
    q = I.quantize_i8(fr["llr"])
    perms = I.perm_table(m, r, P, L, seed=8)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(best, ref["best"])


@pytest.mark.parametrize("algo,kernel", [("pfht", "warp"), ("pfht", "path"), ("autssc", None)])
def test_non_finite_llrs_give_in_range_results_and_leave_other_frames_alone(algo, kernel):
    """Frames holding NaN or infinite LLRs have no meaningful decision, but they must still
    return one of the decoders' codewords with an in-range winner index, and the other frames
    of the batch must decode exactly as without them (both p-FHT-FSCL kernels)."""
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 64, 2.0, seed=71)
    x = fr["llr"].astype(np.float32)
    dec = pkg.Decoder(m, r, P, L, perm_seed=3, algo=algo)
    if kernel is not None:
        dec.set_kernel(kernel)
    ref_info, ref_cw, ref_pm, ref_best = _gpu_decode(dec, x)
    bad = x.copy()
    bad[5, :] = np.nan
    bad[9, 3] = np.inf
    bad[12, :] = np.inf
    bad[12, ::2] = -np.inf
    bad[20, 7] = np.nan
    info, cw, pm, best = _gpu_decode(dec, bad)
    hit = [5, 9, 12, 20]
    assert np.all((best >= 0) & (best < P))
    for f in hit:  # a codeword of RM(2,7): its information bits re-encode to it
        assert np.array_equal(I.encode(info[f:f + 1], m, r)[0], cw[f])
    keep = np.setdiff1d(np.arange(64), hit)
    assert np.array_equal(cw[keep], ref_cw[keep]) and np.array_equal(best[keep], ref_best[keep])


@pytest.mark.parametrize("m,r", [(2, 1), (3, 1), (5, 1), (7, 1), (9, 1), (10, 1), (3, 2), (4, 3), (6, 5), (9, 8),
                                 (10, 9)])
@pytest.mark.parametrize("P,L", [(1, 1), (3, 16)])
def test_first_order_and_parity_check_roots_match_the_oracle(m, r, P, L):
    """RM(1, m) and RM(m-1, m), whose root is an FHTL or SPCL node: INT8 codes bit-exact
    against the integer oracle (word, metric, winner; ties are frequent on the coarse codes),
    FP32 LLRs to the same words with metrics within 1e-5 relative."""
    fr = I.make_frames(m, r, 333, 1.0, seed=90 + m)
    perms = I.perm_table(m, r, P, L, seed=5)
    q = I.quantize_i8(fr["llr"] * 0.5)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True, want_margin=False)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(info, ref["info"]) and np.array_equal(cw, ref["cw"])
    assert np.array_equal(pm.astype(np.int64), ref["pm"]) and np.array_equal(best, ref["best"])
    ref = O.decode(m, r, P, L, perms, fr["llr"])
    dec.set_dtype("f32")
    info, cw, pm, best = _gpu_decode(dec, fr["llr"].astype(np.float32))
    diff = np.any(cw != ref["cw"], axis=1)
    assert np.all(ref["margin"][diff] < 1e-5)  # only FP32 near-ties may decide otherwise
    np.testing.assert_allclose(pm[~diff], ref["pm"][~diff], rtol=1e-5, atol=1e-5 * np.mean(np.abs(fr["llr"])))


@pytest.mark.parametrize("m,r,P,L", [(9, 2, 20, 4), (9, 3, 16, 8), (9, 3, 4, 4), (9, 2, 3, 8)])
def test_tensor_core_hadamard_is_exact_on_small_integer_llrs(m, r, P, L):
    """The tensor-core transform rounds its operands to FP16, which holds every integer up to
    2048 exactly. With INT8 codes within +-64 every FHT operand (|alpha| <= 2^(9-s) 64 at a
    node of 2^s points) and the intermediate H_16 X (<= 32 x 64) stay below that, so the
    variant must then equal the integer oracle bit for bit: this checks the MMA fragment
    layouts and the Kronecker factorisation."""
    fr = I.make_frames(m, r, 400, 2.0, seed=120 + r * 10 + L)
    perms = I.perm_table(m, r, P, L, seed=9)
    q = np.clip(I.quantize_i8(fr["llr"] * 0.6), -64, 64).astype(np.int8)
    ref = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True, want_margin=False)
    dec = pkg.Decoder(m, r, P, L, dtype="i8", perms=perms)
    dec.set_hadamard("tensor")
    info, cw, pm, best = _gpu_decode(dec, q)
    assert np.array_equal(cw, ref["cw"]) and np.array_equal(pm.astype(np.int64), ref["pm"])
    assert np.array_equal(best, ref["best"]) and np.array_equal(info, ref["info"])


def test_tensor_core_hadamard_on_fp16_llrs_decides_like_fp32():
    """RM(3,9), P = 16, L = 8 on FP16 LLRs. With the tensor-core
    transform the decisions may differ from the FP32 butterflies only where FP16 rounding moves
    a candidate; on these frames they differ on at most 1% and the path metric stays within
    1e-2 relative of the returned word's discrepancy."""
    m, r, P, L = 9, 3, 16, 8
    fr = I.make_frames(m, r, 600, 2.5, seed=131)
    perms = I.perm_table(m, r, P, L, seed=2)
    x = I.to_f16(fr["llr"])
    dec = pkg.Decoder(m, r, P, L, dtype="f16", perms=perms)
    ref_info, ref_cw, _, _ = _gpu_decode(dec, x)
    dec.set_hadamard("tensor")
    info, cw, pm, best = _gpu_decode(dec, x)
    diff = np.mean(np.any(cw != ref_cw, axis=1))
    assert diff <= 0.01, diff
    y = x.astype(np.float64)
    np.testing.assert_allclose(pm, _disc(y, cw), rtol=1e-2, atol=1e-2 * np.mean(np.abs(y)))
    nl = I.noiseless_frames(m, r, 20, seed=3)
    ni, _, _, _ = _gpu_decode(dec, I.to_f16(nl["llr"]))
    assert np.array_equal(ni, nl["u"])
    dec.set_hadamard("shuffle")  # and back
    assert np.array_equal(_gpu_decode(dec, x)[1], ref_cw)

