"""Grouped multi-code launches (include/rmdec_group.h) on the GPU, through the C ABI.

One launch decodes segments of several decoders (codes, P, LLR types) at once. Integer LLRs
must match the oracle's exact integer decoder bit for bit; real-valued LLRs must give exactly
what each decoder's own rmdec_decode gives (the arithmetic per frame is the same), whatever
the segment order, sizes and launch splitting.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402

MEMBERS = [  # (m, r, P, dtype, algo): one list size per group
    (7, 2, 8, "i8", "pfht"),
    (9, 2, 20, "f32", "pfht"),   # F32 holding integer codes: exact as well
    (9, 3, 4, "i16", "pfht"),
    (8, 2, 1, "i8", "fhtfscl"),
    (5, 3, 3, "i8", "pfht"),
    (4, 2, 2, "f32", "pfht"),
]


def _members(L, seed):
    decs, perms = [], []
    for i, (m, r, P, dt, algo) in enumerate(MEMBERS):
        if algo == "pfht":
            pt = I.perm_table(m, r, P, L, seed=seed + i)
            decs.append(pkg.Decoder(m, r, P, L, dtype=dt, perms=pt))
        else:
            pt = None
            decs.append(pkg.Decoder(m, r, 1, L, algo="fhtfscl", dtype=dt))
        perms.append(pt)
    return decs, perms


def _as_dtype(dt, q):
    """Integer LLR codes q in a decoder's input type."""
    return {"i8": q.astype(np.int8), "i16": q.astype(np.int16), "f32": q.astype(np.float32)}[dt]


@pytest.mark.parametrize("L", [8, 4, 2, 1])
def test_mixed_group_matches_integer_oracle(L):
    decs, perms = _members(L, seed=40 + L)
    grp = pkg.Group(decs)
    # caller order mixes light and heavy segments, with ragged, single-frame and empty ones
    sizes = [(0, 37), (1, 61), (2, 1), (3, 90), (4, 5), (5, 44), (1, 0), (0, 130), (2, 23), (1, 9)]
    segs, refs = [], []
    for q, (di, nf) in enumerate(sizes):
        m, r, P, dt, algo = MEMBERS[di]
        fr = I.make_frames(m, r, max(nf, 1), 2.0 + 0.3 * q, seed=700 + 13 * q + L)
        codes = I.quantize_i8(fr["llr"])[:nf]
        if dt == "i16":
            codes = codes.astype(np.int16) * 3  # wider codes, still far below the exactness bound
        x = torch.from_numpy(np.ascontiguousarray(_as_dtype(dt, codes))).cuda()
        segs.append((di, x, None))
        if nf == 0:
            refs.append(None)
        elif algo == "pfht":
            refs.append(O.decode(m, r, P, L, perms[di], codes.astype(np.int64), integer=True)["info"])
        else:
            refs.append(O.decode_fhtfscl(m, r, L, codes.astype(np.int64), integer=True)["info"])
    outs = grp.decode(segs)
    torch.cuda.synchronize()
    for q, (out, ref) in enumerate(zip(outs, refs)):
        if ref is None:
            assert out.shape[0] == 0
            continue
        got = pkg.unpack_bits(out.cpu().numpy(), decs[sizes[q][0]].k)
        assert np.array_equal(got, ref), q
    grp.close()


def test_real_valued_group_equals_separate_decodes():
    L = 4
    decs = [pkg.Decoder(7, 2, 8, L, perm_seed=1), pkg.Decoder(8, 2, 8, L, perm_seed=2),
            pkg.Decoder(9, 2, 20, L, perm_seed=3), pkg.Decoder(9, 3, 8, L, perm_seed=4, dtype="f16"),
            pkg.Decoder(6, 2, 4, L, perm_seed=5)]
    grp = pkg.Group(decs)
    segs = []
    rng = np.random.default_rng(9)
    for q in range(14):
        di = int(rng.integers(len(decs)))
        d = decs[di]
        nf = int(rng.integers(1, 400))
        fr = I.make_frames(d.m, d.r, nf, float(rng.uniform(1.5, 4.0)), seed=900 + q)
        x = fr["llr"].astype(np.float16 if di == 3 else np.float32)
        segs.append((di, torch.from_numpy(x).cuda(), None))
    outs = grp.decode(segs)
    for (di, x, _), out in zip(segs, outs):
        assert torch.equal(out, decs[di].decode(x))
    # a different launch shape never changes results (narrow, and wider than some members' P)
    for wq, cq in ((2, 1), (12, 0)):
        grp.set_tuning(wq, cq)
        outs2 = grp.decode(segs)
        assert all(torch.equal(a, b) for a, b in zip(outs, outs2)), (wq, cq)
    grp.close()


@pytest.mark.parametrize("split", [0, -1, 1000])
def test_large_segments_in_own_launches_give_the_same_bits(split):
    decs = [pkg.Decoder(7, 2, 8, 4, perm_seed=1, dtype="i8"), pkg.Decoder(9, 2, 20, 4, perm_seed=2),
            pkg.Decoder(8, 2, 8, 4, perm_seed=3)]
    grp = pkg.Group(decs)
    grp.set_split(split)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    segs = []
    for di, nf in [(0, 5000), (1, 300), (2, 1200), (0, 40), (1, 1600)]:
        d = decs[di]
        _, llr = I.make_frames_torch(d.m, d.r, nf, 2.5, gen)
        x = torch.clamp(torch.round(llr / 0.25), -127, 127).to(torch.int8) if di == 0 else llr
        segs.append((di, x.contiguous(), None))
    outs = grp.decode(segs)
    for (di, x, _), out in zip(segs, outs):
        assert torch.equal(out, decs[di].decode(x))
    grp.close()


def test_long_segment_lists_are_split_over_launches():
    decs = [pkg.Decoder(5, 2, 4, 2, perm_seed=1, dtype="i8"), pkg.Decoder(7, 2, 3, 2, perm_seed=2, dtype="i8")]
    grp = pkg.Group(decs)
    rng = np.random.default_rng(4)
    segs = []
    for q in range(500):  # more segments than one launch carries
        di = q % 2
        d = decs[di]
        nf = int(rng.integers(1, 4))
        fr = I.make_frames(d.m, d.r, nf, 2.5, seed=3000 + q)
        segs.append((di, torch.from_numpy(I.quantize_i8(fr["llr"])).cuda(), None))
    outs = grp.decode(segs)
    for (di, x, _), out in zip(segs, outs):
        assert torch.equal(out, decs[di].decode(x))
    grp.close()


def test_group_launch_replays_from_a_cuda_graph():
    decs = [pkg.Decoder(7, 2, 8, 4, perm_seed=6, dtype="i8"), pkg.Decoder(9, 2, 20, 4, perm_seed=7)]
    grp = pkg.Group(decs)
    f7 = I.make_frames(7, 2, 300, 2.0, seed=1)
    f9 = I.make_frames(9, 2, 200, 2.25, seed=2)
    x7 = torch.from_numpy(I.quantize_i8(f7["llr"])).cuda()
    x9 = torch.from_numpy(f9["llr"].astype(np.float32)).cuda()
    o7 = torch.zeros((300, decs[0].kw), dtype=torch.int32, device="cuda")
    o9 = torch.zeros((200, decs[1].kw), dtype=torch.int32, device="cuda")
    grp.decode([(0, x7, o7), (1, x9, o9)])  # uploads the tables before capture
    torch.cuda.synchronize()
    ref7, ref9 = o7.clone(), o9.clone()
    o7.zero_()
    o9.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            grp.decode([(0, x7, o7), (1, x9, o9)])
    for _ in range(2):
        o7.zero_()
        o9.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(o7, ref7) and torch.equal(o9, ref9)
    assert torch.equal(ref7, decs[0].decode(x7)) and torch.equal(ref9, decs[1].decode(x9))
    grp.close()
