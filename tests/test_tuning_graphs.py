"""Launch-shape tuning, the autotuner's cache and captured CUDA graphs: none of them may change
a single decoded bit."""
import os

import numpy as np
import pytest

import paper_2108_12550_gb300 as pkg
from paper_2108_12550_gb300 import inputs as I

torch = pytest.importorskip("torch")


def test_tuning_arguments_are_validated():
    d = pkg.Decoder(9, 2, 20, 4)
    for bad in [(21, 0), (-1, 0), (2, 33)]:
        with pytest.raises(pkg.RmdecError):
            d.set_tuning(*bad)
    d.set_tuning(2, 1)


@pytest.mark.gpu
@pytest.mark.parametrize("m,r,P,L,ws", [(9, 2, 20, 4, (1, 2, 4, 7, 10, 20)), (9, 3, 16, 8, (1, 2, 4, 8)),
                                        (5, 2, 4, 2, (1, 2, 4, 16))])
def test_every_launch_shape_gives_identical_results(m, r, P, L, ws):
    fr = I.make_frames(m, r, 1000, 2.5, seed=4)
    x = torch.from_numpy(fr["llr"].astype(np.float32)).cuda()
    d = pkg.Decoder(m, r, P, L, perm_seed=3)
    outs = []
    for w in ws:
        for c in (0, 1):
            d.set_tuning(w, c)
            outs.append(d.decode(x).cpu())
            assert d.get_tuning()[0] == min(w, P)
    assert all(torch.equal(o, outs[0]) for o in outs)


@pytest.mark.gpu
def test_autotune_and_cache(tmp_path):
    cache = str(tmp_path / "tune.txt")
    d = pkg.Decoder(9, 2, 20, 4, perm_seed=1)
    w, c = d.autotune(n_frames=8192, cache_path=cache)
    assert 1 <= w <= 20 and c >= 1
    lines = open(cache).read().split("\n")
    assert len([l for l in lines if l.strip()]) == 1
    d2 = pkg.Decoder(9, 2, 20, 4, perm_seed=2)
    assert d2.autotune(n_frames=8192, cache_path=cache)[0] == w  # reused, not re-timed
    assert len([l for l in open(cache).read().split("\n") if l.strip()]) == 1


@pytest.mark.gpu
def test_graph_replays_match_direct_decoding():
    m, r, P, L = 7, 2, 8, 4
    d = pkg.Decoder(m, r, P, L, perm_seed=6)
    fr = I.make_frames(m, r, 777, 2.0, seed=8)
    host_in = torch.from_numpy(fr["llr"].astype(np.float32)).pin_memory()
    host_out = torch.zeros((777, d.kw), dtype=torch.int32).pin_memory()
    ref = d.decode(host_in.cuda()).cpu()
    g = d.graph(host_in, host_out)
    for _ in range(3):
        host_out.zero_()
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(host_out, ref)
    # new LLRs in the same host buffer are picked up by the next replay
    fr2 = I.make_frames(m, r, 777, 2.0, seed=9)
    host_in.copy_(torch.from_numpy(fr2["llr"].astype(np.float32)))
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(host_out, d.decode(host_in.cuda()).cpu())
    g.close()


@pytest.mark.gpu
def test_graph_replay_after_new_permutations_uses_the_new_tables():
    """rmdec_set_perms followed by a decode overwrites the handle's device tables in place, so
    a graph captured before still reads valid memory and decodes with the new permutations."""
    m, r, P, L = 7, 2, 1, 1  # a single decoder at 1 dB: its decisions depend on its table
    d = pkg.Decoder(m, r, P, L, perm_seed=6)
    fr = I.make_frames(m, r, 500, 1.0, seed=18)
    host_in = torch.from_numpy(fr["llr"].astype(np.float32)).pin_memory()
    host_out = torch.zeros((500, d.kw), dtype=torch.int32).pin_memory()
    old = d.decode(host_in.cuda()).cpu()
    g = d.graph(host_in, host_out)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(host_out, old)
    d.set_perms(I.perm_table(m, r, P, L, seed=77))
    new = d.decode(host_in.cuda()).cpu()  # uploads the new tables
    other = pkg.Decoder(m, r, P, L, perms=I.perm_table(m, r, P, L, seed=77))
    assert torch.equal(new, other.decode(host_in.cuda()).cpu())
    assert not torch.equal(new, old)  # the tables differ in effect on these frames
    host_out.zero_()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(host_out, new)
    g.close()
    other.close()


@pytest.mark.gpu
@pytest.mark.parametrize("m,r,P,L", [(9, 2, 20, 4), (7, 2, 8, 4), (9, 3, 16, 8)])
def test_launch_size_never_changes_results(m, r, P, L):
    """Launches of a few waves run in wider shapes than large ones; every frame must decode
    the same whatever batch it is part of."""
    d = pkg.Decoder(m, r, P, L, perm_seed=9)
    big = 6000
    fr = I.make_frames(m, r, big, 2.5, seed=12)
    x = torch.from_numpy(fr["llr"].astype(np.float32)).cuda()
    ref = d.decode(x).cpu()
    off = 0
    for n in (1, 3, 37, 152, 700, 1500, 3000):
        n = min(n, big - off)
        assert torch.equal(d.decode(x[off:off + n]).cpu(), ref[off:off + n]), n
        off += n


@pytest.mark.gpu
def test_large_host_decode_in_chunks_matches_device_decode():
    """rmdec_decode_host splits batches of 16+ waves into chunks whose uploads overlap the
    previous chunk's decode; the bits must equal one device-resident decode."""
    m, r, P, L = 5, 2, 4, 2
    d = pkg.Decoder(m, r, P, L, perm_seed=13)
    w, c = d.get_tuning()
    n = 40 * 152 * c + 123  # more than 32 waves of the default shape on a 152-SM GPU, ragged
    fr = I.make_frames(m, r, 4096, 3.0, seed=14)
    x = np.tile(fr["llr"].astype(np.float32), (n // 4096 + 1, 1))[:n]
    host_in = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    host_out = torch.zeros((n, d.kw), dtype=torch.int32).pin_memory()
    d.decode_host(host_in, host_out)
    ref = d.decode(host_in.cuda()).cpu()
    assert torch.equal(host_out, ref)
