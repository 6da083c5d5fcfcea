"""Pins of the CPU oracle to facts fixed by the paper and by mathematics, independent of the
oracle's own code: a library Hadamard matrix, closed-form FHT spectra, brute-force maximum
likelihood on small codes, the path-metric = discrepancy identity, noiseless decoding, the
integer mode, the permutation selection on inputs whose reliability order is fixed by
construction, and the frame error rates printed in the paper's figures."""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2108_12550_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _disc(llr, cw):
    """Correlation discrepancy sum_i |y_i| [x_i != HD(y_i)] (the long path metric, Eq. (7))."""
    return np.sum(np.abs(llr) * (cw != (llr < 0)), axis=-1)


# ------------------------------------------------------------------ FHT (Algorithm 4) ---

@pytest.mark.parametrize("s", [1, 2, 3, 5, 8])
def test_fht_equals_sylvester_hadamard_product(s):
    rng = np.random.default_rng(s)
    a = rng.normal(size=1 << s)
    # scipy's Sylvester matrix has H[k, j] = (-1)^popcount(k & j)
    np.testing.assert_allclose(O.fht(a), scipy.linalg.hadamard(1 << s) @ a, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("s", [3, 6, 8])
def test_fht_of_noiseless_first_order_word_has_single_peak(s):
    n = 1 << s
    j = np.arange(n)
    for k in [0, 1, n - 1, n // 3]:
        for sign in [0, 1]:
            x = (np.array([bin(k & v).count("1") & 1 for v in j]) ^ sign)
            c = O.fht(1.0 - 2.0 * x)
            assert abs(c[k]) == n and (c[k] < 0) == bool(sign)
            assert np.count_nonzero(c) == 1


def _rm1_codewords(s):
    n = 1 << s
    j = np.arange(n)
    words = []
    for k in range(n):
        base = np.array([bin(k & v).count("1") & 1 for v in j], dtype=np.uint8)
        words.append((k, 0, base))
        words.append((k, 1, base ^ 1))
    return words


@pytest.mark.parametrize("s", [3, 4, 6])
def test_fhtl_single_path_is_ml_and_top_list_by_brute_force(s):
    rng = np.random.default_rng(10 + s)
    words = _rm1_codewords(s)
    for trial in range(20):
        a = rng.normal(size=(1, 1 << s)) * 2
        # L = 1: FHT decoding is maximum likelihood for RM(1, s)
        _, x, pm = O.fhtl(a, np.zeros(1))
        d = [(_disc(a[0], w), k, sg) for k, sg, w in words]
        best = min(d)
        assert abs(pm[0] - best[0]) < 1e-9 and abs(_disc(a[0], x[0]) - best[0]) < 1e-9
        # L = 4: the list holds the 4 best codewords among "best sign per index k"
        L = 4
        _, x4, pm4 = O.fhtl(np.repeat(a, 1, axis=0).repeat(1, axis=0)[:1].repeat(L, axis=0) * 0 + a,
                             np.array([0.0, 1e9, 1e9, 1e9]))
        per_k = {}
        for dv, k, sg in d:
            per_k[k] = min(per_k.get(k, (np.inf,)), (dv, k, sg))
        expect = sorted(per_k.values())[:L]
        np.testing.assert_allclose(pm4, [e[0] for e in expect], atol=1e-9)
        for q in range(L):
            assert abs(_disc(a[0], x4[q]) - pm4[q]) < 1e-9  # Eq. (7) = Eq. (8)


def _even_words(n):
    out = []
    for v in range(1 << n):
        w = np.array([(v >> i) & 1 for i in range(n)], dtype=np.uint8)
        if w.sum() % 2 == 0:
            out.append(w)
    return np.array(out)


@pytest.mark.parametrize("s,L", [(3, 1), (3, 2), (3, 4), (3, 8), (4, 1), (4, 4), (4, 8)])
def test_spcl_single_path_lists_the_best_parity_words(s, L):
    """L = 1 is the Wagner rule; with one live path the SPCL list (tau = min(L, N-1)
    splits) is the L most likely even-weight words, found here by enumeration."""
    rng = np.random.default_rng(100 + 7 * s + L)
    words = _even_words(1 << s)
    for trial in range(30):
        a = rng.normal(size=(1, 1 << s)) * 3
        alpha = np.repeat(a, L, axis=0)
        pm0 = np.full(L, 1e9)
        pm0[0] = 0.0  # only path 0 is live
        _, x, pm = O.spcl(alpha, pm0)
        d = np.sort(_disc(a[0], words))
        k = min(L, len(words))
        np.testing.assert_allclose(pm[:k], d[:k], atol=1e-9)
        for q in range(k):
            assert x[q].sum() % 2 == 0 and abs(_disc(a[0], x[q]) - pm[q]) < 1e-9


# ----------------------------------------------------------- whole decoder (Alg. 2-5) ---

CODES = [(4, 2), (5, 2), (5, 3), (6, 2), (6, 3), (7, 2), (9, 2), (9, 3)]


@pytest.mark.parametrize("m,r", CODES)
@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_noiseless_frames_decode_exactly(m, r, L):
    P = 3
    perms = I.perm_table(m, r, P, L, seed=m * 100 + r * 10 + L)
    nl = I.noiseless_frames(m, r, 6, seed=L)
    out = O.decode(m, r, P, L, perms, nl["llr"])
    assert np.array_equal(out["info"], nl["u"]) and np.array_equal(out["cw"], nl["x"])
    assert np.all(np.abs(out["pm"]) < 1e-9)


@pytest.mark.parametrize("m,r,P,L,eb", [(5, 2, 4, 2, 2.0), (7, 2, 8, 4, 2.0), (9, 2, 4, 4, 2.0),
                                        (5, 3, 2, 8, 3.0), (9, 3, 2, 8, 3.0)])
def test_path_metric_equals_discrepancy(m, r, P, L, eb):
    """For min-sum f and exact g the path metric telescopes to the correlation discrepancy of
    the decoded word in the channel domain; permutations preserve it."""
    perms = I.perm_table(m, r, P, L, seed=3)
    fr = I.make_frames(m, r, 60, eb, seed=m + r)
    out = O.decode(m, r, P, L, perms, fr["llr"])
    D = _disc(fr["llr"], out["cw"])
    np.testing.assert_allclose(out["pm"], D, rtol=1e-12, atol=1e-9)
    qi = I.quantize_i8(fr["llr"]).astype(np.int64)
    oi = O.decode(m, r, P, L, perms, qi, integer=True)
    assert np.array_equal(oi["pm"], _disc(qi, oi["cw"]).astype(np.int64))


@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (7, 2, 8, 4), (9, 3, 2, 8)])
def test_integer_mode_equals_fp64_on_integer_llrs(m, r, P, L):
    perms = I.perm_table(m, r, P, L, seed=21)
    fr = I.make_frames(m, r, 80, 1.5, seed=22)
    q = I.quantize_i8(fr["llr"])
    a = O.decode(m, r, P, L, perms, q.astype(np.int64), integer=True)
    b = O.decode(m, r, P, L, perms, q.astype(np.float64))
    assert np.array_equal(a["cw"], b["cw"]) and np.array_equal(a["pm"].astype(np.float64), b["pm"])
    assert np.array_equal(a["best"], b["best"])


@pytest.mark.parametrize("m,r", [(4, 2), (5, 2)])
def test_brute_force_ml(m, r):
    """Exhaustive ML over all 2^K codewords (2^11 for RM(2,4), 2^16 for RM(2,5)): the
    decoder never beats ML, and with a large list it reaches ML on nearly every frame."""
    n, k = I.rm_dims(m, r)
    u = ((np.arange(1 << k)[:, None] >> np.arange(k)) & 1).astype(np.uint8)
    book = I.encode(u, m, r).astype(np.float64)
    fr = I.make_frames(m, r, 300, 1.0, seed=5)
    corr = fr["llr"] @ (1 - 2 * book).T  # maximise correlation = minimise discrepancy
    ml = book[np.argmax(corr, axis=1)].astype(np.uint8)
    d_ml = _disc(fr["llr"], ml)
    P, L = 8, 8
    out = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=9), fr["llr"])
    d_dec = _disc(fr["llr"], out["cw"])
    assert np.all(d_dec >= d_ml - 1e-9)
    hit = np.mean(np.abs(d_dec - d_ml) < 1e-9)
    assert hit >= 0.97, hit
    # a single decoder with L = 1 is clearly weaker than the big list (sanity of the list)
    o1 = O.decode(m, r, 1, 1, I.perm_table(m, r, 1, 1, seed=9), fr["llr"])
    assert np.mean(np.abs(_disc(fr["llr"], o1["cw"]) - d_ml) < 1e-9) < hit


def test_ssc_baseline_properties():
    m, r = 7, 2
    perms = np.stack([I.sample_ga(m, 4, 0, q) for q in range(16)])
    nl = I.noiseless_frames(m, r, 5, seed=2)
    out = O.aut_ssc(m, r, perms, nl["llr"])
    assert np.array_equal(out["info"], nl["u"])
    fr = I.make_frames(m, r, 100, 2.0, seed=8)
    out = O.aut_ssc(m, r, perms, fr["llr"])
    np.testing.assert_allclose(out["disc"], _disc(fr["llr"], out["cw"]), atol=1e-9)
    # more permutations can only lower the selected discrepancy (it is a minimum over them)
    o4 = O.aut_ssc(m, r, perms[:4], fr["llr"])
    assert np.all(out["disc"] <= o4["disc"] + 1e-12)


# ------------------------------- roots that are themselves FHTL / SPCL nodes (Algorithm 2) ---

@pytest.mark.parametrize("m", [2, 3, 5, 7, 9])
@pytest.mark.parametrize("integer", [False, True])
def test_first_order_root_decodes_to_ml_by_enumeration(m, integer):
    """RM(1, m) as a whole code: the root is an FHTL node, so every decoder returns the ML
    word (largest |c_k|, ties to the smaller k, the sign of c_k); enumerating all 2^(m+1)
    codewords in the order (k, sign) and taking the first of smallest discrepancy pins it,
    including the tie rule on integer frames, where ties are frequent."""
    r, P, L = 1, 3, 2
    n = 1 << m
    j = np.arange(n)
    book = np.array([[(bin(k & v).count("1") & 1) ^ sgn for v in j] for k in range(n) for sgn in (0, 1)],
                    dtype=np.uint8)
    fr = I.make_frames(m, r, 300, 0.0, seed=70 + m)
    y = I.quantize_i8(fr["llr"] * 0.3).astype(np.int64) if integer else fr["llr"]
    out = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=3), y, integer=integer, want_margin=False)
    disc = np.stack([_disc(y, np.broadcast_to(w, y.shape)) for w in book], axis=1)
    assert np.array_equal(out["cw"], book[np.argmin(disc, axis=1)])
    assert np.array_equal(out["pm"], disc.min(axis=1)) if integer else np.allclose(out["pm"], disc.min(axis=1))
    assert np.all(out["best"] == 0)  # every decoder decides alike: the first wins
    if integer:
        assert np.mean(np.sum(disc == disc.min(axis=1, keepdims=True), axis=1) > 1) > 0.05  # ties occur


@pytest.mark.parametrize("m", [3, 4, 6, 10])
def test_parity_check_root_decodes_by_wagner_rule(m):
    """RM(m-1, m): the root is an SPCL node; the best path is the hard decision with the least
    reliable bit flipped on odd parity, which is ML (pinned by enumerating the even-weight
    words for m <= 4)."""
    r, P, L = m - 1, 2, 4
    n = 1 << m
    fr = I.make_frames(m, r, 300, 1.0, seed=80 + m)
    out = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=4), fr["llr"], want_margin=False)
    hd = (fr["llr"] < 0).astype(np.uint8)
    a = np.abs(fr["llr"])
    odd = np.sum(hd, axis=1) % 2 == 1
    want = hd.copy()
    want[np.arange(300)[odd], np.argmin(a, axis=1)[odd]] ^= 1
    assert np.array_equal(out["cw"], want)
    np.testing.assert_allclose(out["pm"], np.where(odd, a.min(axis=1), 0.0), rtol=0, atol=1e-12)
    if n <= 16:
        words = ((np.arange(1 << n)[:, None] >> np.arange(n)) & 1).astype(np.uint8)
        book = words[np.sum(words, axis=1) % 2 == 0]
        idx, _ = _ml_by_enumeration(fr["llr"], book)
        assert np.array_equal(out["cw"], book[idx])


# ------------------------------------------- Aut-SSC node rules (repetition, Wagner SPC) ---

def _ml_by_enumeration(llr, book):
    """Smallest correlation discrepancy over an explicit list of codewords; returns the
    index of the first minimiser per frame."""
    disc = np.stack([_disc(llr, w[None, :].repeat(llr.shape[0], 0)) for w in book], axis=1)
    return np.argmin(disc, axis=1), disc


def _identity(m):
    rec = np.zeros((1, I.PERM_REC), dtype=np.uint16)
    rec[0, :m] = 1 << np.arange(m)
    return rec


@pytest.mark.parametrize("m", [3, 5, 8])
def test_ssc_repetition_node_is_ml_on_the_repetition_code(m):
    """RM(0, m) is the repetition code {0^N, 1^N}; SSC decodes it at one repetition node, whose
    rule (the sign of the LLR sum, bit 0 on a zero sum) is ML. Enumerating both codewords pins
    the rule, its sign convention and its tie rule (integer frames with zero sums)."""
    n = 1 << m
    book = np.stack([np.zeros(n, np.uint8), np.ones(n, np.uint8)])
    fr = I.make_frames(m, 0, 400, -2.0, seed=50 + m)
    out = O.aut_ssc(m, 0, _identity(m), fr["llr"])
    idx, disc = _ml_by_enumeration(fr["llr"], book)
    assert np.array_equal(out["cw"], book[idx])
    np.testing.assert_allclose(out["disc"], disc.min(axis=1), rtol=0, atol=1e-9)
    assert 0.05 < np.mean(idx == 1) < 0.95  # both codewords are chosen
    # integer LLRs with exact zero sums: both words have equal discrepancy, bit 0 is chosen
    rng = np.random.default_rng(m)
    q = rng.integers(-3, 4, size=(300, n)).astype(np.int64)
    q[:100, -1] -= q[:100].sum(axis=1)  # the first 100 frames sum to zero
    outi = O.aut_ssc(m, 0, _identity(m), q, integer=True)
    s = q.sum(axis=1)
    assert np.array_equal(outi["cw"][:, 0], (s < 0).astype(np.uint8))
    assert np.all(outi["cw"] == outi["cw"][:, :1])


@pytest.mark.parametrize("m", [3, 4, 6])
def test_ssc_wagner_node_is_ml_on_the_parity_check_code(m):
    """RM(m-1, m) is the even-weight code; SSC decodes it at one SPC node, whose Wagner rule
    (hard decisions, then flip the least reliable bit when the parity is odd) is ML.
    Enumerating every even-weight word pins the rule: the least reliable bit, not another
    one, and flipped only on odd parity."""
    n = 1 << m
    words = ((np.arange(1 << n)[:, None] >> np.arange(n)) & 1).astype(np.uint8) if n <= 16 else None
    fr = I.make_frames(m, m - 1, 400, 0.0, seed=60 + m)
    out = O.aut_ssc(m, m - 1, _identity(m), fr["llr"])
    if words is not None:
        book = words[np.sum(words, axis=1) % 2 == 0]
        idx, disc = _ml_by_enumeration(fr["llr"], book)
        assert np.array_equal(out["cw"], book[idx])
    # any size: the chosen word has even weight and no even-weight word is closer; the
    # best alternatives are the hard decision (odd parity fixed at one position) and, for an
    # even hard decision, the hard decision itself
    hd = (fr["llr"] < 0).astype(np.uint8)
    assert np.all(np.sum(out["cw"], axis=1) % 2 == 0)
    a = np.abs(fr["llr"])
    odd = np.sum(hd, axis=1) % 2 == 1
    best = np.where(odd, a.min(axis=1), 0.0)  # ML discrepancy of the even-weight code
    np.testing.assert_allclose(out["disc"], best, rtol=0, atol=1e-12)
    assert 0.2 < np.mean(odd) < 0.8


def _paper_rows():
    rows = []
    for line in open(os.path.join(GOLD, "paper_fer.txt")):
        if line.strip() and not line.startswith("#"):
            t = line.split()
            rows.append((int(t[0]), int(t[1]), t[2], int(t[3]), int(t[4]), float(t[5]), float(t[6]), " ".join(t[7:])))
    return rows


@pytest.mark.parametrize("row", _paper_rows(), ids=lambda r: r[7].replace(" ", "_") + f"@{r[5]}dB")
def test_fer_matches_paper_figures(row):
    """Monte-Carlo FER against the values printed in the paper's Figs. 4 and 6. The band
    (a factor 2.2 either way) is wide enough for the sample size and for the unstated
    Eb/N0 convention, narrow enough to catch a wrong list rule or a dropped term."""
    m, r, dec, P, L, eb, fer_paper, _ = row
    n_frames = int(min(16000, max(1500, 30 / fer_paper)))  # about 30 expected errors
    fr = I.make_frames(m, r, n_frames, eb, seed=2024)
    if dec == "pfht":
        out = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=31), fr["llr"], want_margin=False)
    elif dec == "fhtfscl":
        out = O.decode_fhtfscl(m, r, L, fr["llr"])
    else:
        perms = np.stack([I.sample_ga(m, 31, 0, q) for q in range(P)])
        out = O.aut_ssc(m, r, perms, fr["llr"])
    errs = int(np.sum(np.any(out["info"] != fr["u"], axis=1)))
    fer = errs / n_frames
    assert fer_paper / 2.2 <= fer <= fer_paper * 2.2, (fer, errs, n_frames, fer_paper)


def _complexity_rows():
    rows = []
    for line in open(os.path.join(GOLD, "paper_complexity.txt")):
        if line.strip() and not line.startswith("#"):
            t = line.split()
            rows.append((int(t[0]), int(t[1]), t[2], int(t[3]), int(t[4]), t[5], " ".join(t[6:])))
    return rows


@pytest.mark.parametrize("row", _complexity_rows(), ids=lambda r: r[6].replace(" ", "_"))
def test_paper_complexity_count_reproduces_printed_values(row):
    """The oracle's count in the paper's convention (floating-point additions and comparisons,
    Section III-C) equals, to the digits printed, the complexity C that Fig. 5 prints for
    FHT-FSCL-1 and p-FHT-FSC-1 on RM(2|3|4, 9) and that Table 5 prints for p-FHT-FSCL-1-M1 on
    RM(2|3|4, 8) and RM(2, 9). Every term of the L = 1 count enters: f and g (one per
    output), the FHT's s 2^s additions, the SPC node's 2^s, and each permuted node's 2L 2^(s-1)
    reliability evaluations plus the 2L log2(2L) sort; C is P times the count of one decoder.
    A dropped, doubled or misplaced term moves at least one of the ten values."""
    m, r, dec, P, L, printed, _ = row
    fr = I.make_frames(m, r, 2, 3.0, seed=17)
    if dec == "fhtfscl":
        ops, paper = O.op_counts(m, r, 1, L, None, fr["llr"], no_perm=True)
    else:
        ops, paper = O.op_counts(m, r, P, L, I.perm_table(m, r, P, L, seed=17), fr["llr"])
    assert paper[0] == paper[1]  # the count depends on the code, not on the frame
    mant = printed.upper().split("E")[0]
    digits = len(mant.replace(".", "").lstrip("0"))
    got = f"{float(paper[0]):.{digits - 1}E}"
    assert float(got) == float(printed), (int(paper[0]), got, printed)
    # this build's count (the roofline numerator) holds every term of the paper's count
    assert np.all(ops > paper)


@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (7, 2, 8, 4), (9, 2, 20, 4), (9, 3, 16, 8), (6, 3, 2, 1)])
def test_operation_count_model_matches_oracle_counter(m, r, P, L):
    from paper_2108_12550_gb300 import opcount

    fr = I.make_frames(m, r, 2, 2.0, seed=1)
    o = O.decode(m, r, P, L, I.perm_table(m, r, P, L, seed=1), fr["llr"], want_ops=True)
    assert np.all(o["ops"] == opcount.ops_per_frame(m, r, P, L))


@pytest.mark.parametrize("m,r,L", [(5, 2, 1), (7, 2, 4), (9, 3, 8)])
def test_fhtfscl_is_the_permuted_decoder_with_identity_permutations(m, r, L):
    """FHT-FSCL equals p-FHT-FSCL when every permutation is the identity and only one initial
    path is live: checked on L = 1, where both start from a single path."""
    fr = I.make_frames(m, r, 200, 2.0, seed=3)
    a = O.decode_fhtfscl(m, r, L, fr["llr"])
    D = _disc(fr["llr"], a["cw"])
    np.testing.assert_allclose(a["pm"], D, rtol=1e-12, atol=1e-9)  # metric = discrepancy
    nl = I.noiseless_frames(m, r, 8, seed=1)
    assert np.array_equal(O.decode_fhtfscl(m, r, L, nl["llr"])["info"], nl["u"])
    if L == 1:
        ident = np.zeros((1, I.perms_per_decoder(m, r, 1), I.PERM_REC), dtype=np.uint16)
        for q in range(ident.shape[1]):
            s = m if q < 1 else m - (q - 1) // 2
            ident[0, q, :s] = 1 << np.arange(s)
        b = O.decode(m, r, 1, 1, ident, fr["llr"])
        assert np.array_equal(a["cw"], b["cw"])
    q = I.quantize_i8(fr["llr"]).astype(np.int64)
    ai = O.decode_fhtfscl(m, r, L, q, integer=True)
    assert np.array_equal(ai["pm"], _disc(q, ai["cw"]).astype(np.int64))


# ------------------------------------------- permutation selection (Algorithm 2) ---

@pytest.mark.parametrize("level", ["root", "deeper"])
@pytest.mark.parametrize("integer", [False, True])
def test_selection_keeps_the_more_reliable_permutation_and_breaks_ties_by_index(level, integer):
    """With L = 1 the path extension keeps the one of two candidate permutations whose left
    child has the larger LM = sum |f| (Algorithm 2, the paper's 'maximum channel reliability'),
    the earlier candidate on equal LM. For an affine map the left child pairs positions
    {j, j xor a}, a the image of the top index bit, so LM depends on the map only through a,
    and inputs.selection_case fixes its order by construction: LM(a = 16) = 14 large + 2 small
    terms > LM(a = 1) = 12 large + 4 small terms (A and A2 share a = 16: equal LM). The decode
    must then equal the decode whose two candidates are both the winner."""
    c = I.selection_case(level, 1500, seed=11, integer=integer)
    m, r, y = c["m"], c["r"], c["llr"]
    if integer:
        y = y.astype(np.int64)

    def dec(c0, c1):
        return O.decode(m, r, 1, 1, np.stack(c["head"] + [c0, c1])[None], y, integer=integer, want_margin=False)

    def same(p, q):
        return np.all(p["cw"] == q["cw"], axis=1) & (p["pm"] == q["pm"])

    A, A2, B = c["A"], c["A2"], c["B"]
    aa, bb, a2a2 = dec(A, A), dec(B, B), dec(A2, A2)
    # larger LM wins, in either candidate order
    assert np.all(same(dec(A, B), aa)) and np.all(same(dec(B, A), aa))
    # equal LM: the earlier candidate wins
    assert np.all(same(dec(A, A2), aa)) and np.all(same(dec(A2, A), a2a2))
    # the checks have power: the three maps decide differently on many frames
    assert np.mean(np.any(bb["cw"] != aa["cw"], axis=1)) > 0.2
    assert np.mean(np.any(a2a2["cw"] != aa["cw"], axis=1)) > 0.2


# ----------------------------------------------------- best of P decoders (Algorithm 5) ---

@pytest.mark.parametrize("integer", [False, True])
def test_best_of_p_decoders_is_the_smallest_metric_earliest_on_ties(integer):
    """The P decoders are independent (Algorithm 5): decoding with P tables must return, per
    frame, the result of the decoder whose own run (P = 1, its table alone) has the smallest
    path metric, the earliest such decoder on equal metrics. Decoder 2 repeats decoder 0's
    table, so the two tie exactly on every frame and decoder 2 must never be chosen."""
    m, r, P, L = 7, 2, 4, 2
    tab = I.perm_table(m, r, P, L, seed=23)
    tab[2] = tab[0]
    fr = I.make_frames(m, r, 800, 1.5, seed=41)
    y = I.quantize_i8(fr["llr"]).astype(np.int64) if integer else fr["llr"]
    allp = O.decode(m, r, P, L, tab, y, integer=integer, want_margin=False)
    alone = [O.decode(m, r, 1, L, tab[p:p + 1], y, integer=integer, want_margin=False) for p in range(P)]
    pms = np.stack([a["pm"] for a in alone])          # (P, F)
    want = np.argmin(pms, axis=0)                     # first index of the minimum
    assert np.array_equal(allp["best"], want)
    assert np.array_equal(allp["pm"], pms.min(axis=0))
    for p in range(P):
        sel = want == p
        assert np.array_equal(allp["cw"][sel], alone[p]["cw"][sel])
    assert not np.any(allp["best"] == 2)
    # power: several decoders win somewhere, and decoder 0 (tied with 2) wins often
    assert len(set(want.tolist())) >= 3 and np.mean(want == 0) > 0.2
