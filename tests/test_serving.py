"""Continuous-batching server (include/rmdec_serve.h): results are the same alone and in the
mix, admission waits for device memory, and bad requests are rejected on the host."""
import threading

import numpy as np
import pytest

import paper_2108_12550_gb300 as pkg
from paper_2108_12550_gb300 import inputs as I

torch = pytest.importorskip("torch")

MIX = [  # (m, r, P, L, dtype, algo)
    (7, 2, 8, 4, "i8", "pfht"),
    (8, 2, 8, 4, "f32", "pfht"),
    (9, 2, 20, 4, "f32", "pfht"),
    (9, 3, 8, 4, "i8", "pfht"),
    (7, 2, 16, 1, "f32", "autssc"),  # never fused: decoded by its own launches
]


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n):
        c = int(rng.integers(len(MIX)))
        m, r, P, L, dt, _ = MIX[c]
        nf = int(np.exp(rng.uniform(0, np.log(300))))
        fr = I.make_frames(m, r, nf, float(rng.uniform(2, 5)), seed=seed * 1000 + q)
        x = I.quantize_i8(fr["llr"]) if dt == "i8" else fr["llr"].astype(np.float32)
        reqs.append((c, torch.from_numpy(x).pin_memory()))
    return reqs


@pytest.mark.gpu
@pytest.mark.parametrize("fuse", [False, True])
def test_mixed_requests_match_alone_decoding(fuse):
    decs = [pkg.Decoder(m, r, P, L, perm_seed=11 + i, dtype=dt, algo=algo)
            for i, (m, r, P, L, dt, algo) in enumerate(MIX)]
    reqs = _requests(120, seed=3 + fuse)
    # alone: one decode call per request
    alone = [decs[c].decode(x.cuda()).cpu() for c, x in reqs]
    srv = pkg.Server(n_streams=4, arena_bytes=64 << 20, max_batch_frames=4096, min_batch_frames=256,
                     max_wait_us=200, fuse_codes=fuse)
    ids = [srv.add_decoder(d) for d in decs]
    outs = [torch.zeros((x.shape[0], decs[c].kw), dtype=torch.int32).pin_memory() for c, x in reqs]
    rids = [None] * len(reqs)

    def submit(lo, hi):
        for q in range(lo, hi):
            c, x = reqs[q]
            rids[q] = srv.submit(ids[c], x, outs[q])

    th = [threading.Thread(target=submit, args=(0, 60)), threading.Thread(target=submit, args=(60, 120))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for q, rid in enumerate(rids):
        st, lat = srv.poll(rid, timeout_us=30_000_000)
        assert st == pkg.OK and lat > 0
        assert torch.equal(outs[q], alone[q]), q
    s = srv.stats()
    assert s["completed"] == 120 and s["queued"] == 0 and s["in_flight"] == 0
    assert 0 < s["batches"] <= 120 and s["latency_p50_us"] <= s["latency_p99_us"]
    srv.close()


@pytest.mark.gpu
def test_batches_never_exceed_the_arena():
    """Requests that fit the arena one at a time but not together (arena for one and a half,
    batch cap for all three) are admitted in arena-sized batches instead of waiting for a
    batch that could never fit. A slower request on the only stream makes the three queue
    together before the first batch is formed."""
    dec = pkg.Decoder(9, 2, 4, 4, perm_seed=2)
    slow = pkg.Decoder(9, 3, 16, 8, perm_seed=3, dtype="f16")
    one = 2048 * 512 * 4 + 2048 * 8  # LLRs and output words of one 2048-frame RM(2,9) request
    srv = pkg.Server(n_streams=1, arena_bytes=one * 3 // 2, max_batch_frames=1 << 16)
    cid, sid = srv.add_decoder(dec), srv.add_decoder(slow)
    fs = I.make_frames(9, 3, 2048, 4.0, seed=5)
    xs_slow = torch.from_numpy(I.to_f16(fs["llr"])).pin_memory()
    out_slow = torch.zeros((2048, slow.kw), dtype=torch.int32).pin_memory()
    fr = I.make_frames(9, 2, 2048, 3.0, seed=4)
    xs = [torch.from_numpy(fr["llr"].astype(np.float32)).pin_memory() for _ in range(3)]
    outs = [torch.zeros((2048, 2), dtype=torch.int32).pin_memory() for _ in range(3)]
    rid_slow = srv.submit(sid, xs_slow, out_slow)
    rids = [srv.submit(cid, x, o) for x, o in zip(xs, outs)]
    for rid in [rid_slow] + rids:
        assert srv.poll(rid, timeout_us=30_000_000)[0] == pkg.OK
    ref = dec.decode(xs[0].cuda()).cpu()
    assert all(torch.equal(o, ref) for o in outs)
    assert torch.equal(out_slow, slow.decode(xs_slow.cuda()).cpu())
    assert srv.stats()["batches"] == 4
    srv.close()


@pytest.mark.gpu
def test_admission_waits_for_arena_memory_and_rejects_oversize():
    dec = pkg.Decoder(9, 2, 4, 4, perm_seed=2)
    # room for one 2048-frame batch of RM(2,9) FP32 LLRs (4 MiB + outputs)
    srv = pkg.Server(n_streams=4, arena_bytes=(4 << 20) + (64 << 10), max_batch_frames=2048)
    cid = srv.add_decoder(dec)
    fr = I.make_frames(9, 2, 2048, 3.0, seed=1)
    xs = [torch.from_numpy(fr["llr"].astype(np.float32)).pin_memory() for _ in range(5)]
    outs = [torch.zeros((2048, 2), dtype=torch.int32).pin_memory() for _ in range(5)]
    rids = [srv.submit(cid, x, o) for x, o in zip(xs, outs)]
    for rid in rids:
        assert srv.poll(rid, timeout_us=30_000_000)[0] == pkg.OK
    ref = dec.decode(xs[0].cuda()).cpu()
    assert all(torch.equal(o, ref) for o in outs)
    assert srv.stats()["batches"] == 5  # each batch had to wait for the previous one's memory
    big = torch.zeros((4096, 512), dtype=torch.float32).pin_memory()
    with pytest.raises(pkg.RmdecError) as ei:
        srv.submit(cid, big, torch.zeros((4096, 2), dtype=torch.int32))
    assert ei.value.status == pkg.EINVAL
    with pytest.raises(pkg.RmdecError):
        srv.poll(123456789, 0)
    with pytest.raises(pkg.RmdecError):
        srv.submit(7, xs[0], outs[0])  # unknown code
    srv.close()


def test_server_configuration_is_validated_on_the_host():
    lib = pkg._load_server_api(pkg.load_library())
    import ctypes

    h = ctypes.c_void_p()
    bad = pkg._ServerConfig(0, 1 << 20, 16, 0, 0)
    assert lib.rmdec_server_create(ctypes.byref(h), ctypes.byref(bad)) == pkg.EINVAL
    bad = pkg._ServerConfig(2, 1 << 20, 16, 0, 0, 2)  # fuse_codes is 0 or 1
    assert lib.rmdec_server_create(ctypes.byref(h), ctypes.byref(bad)) == pkg.EINVAL
    assert lib.rmdec_server_create(ctypes.byref(h), None) == pkg.EINVAL
    if not torch.cuda.is_available():
        ok = pkg._ServerConfig(2, 1 << 20, 16, 0, 0)
        st = lib.rmdec_server_create(ctypes.byref(h), ctypes.byref(ok))
        assert st in (pkg.EDEVICE, pkg.ENOMEM) and h.value is None
