"""Failure handling made on the host: injected device-allocation failures surface as
RMDEC_ENOMEM and leave every handle usable; requests cancelled before admission are retired
with RMDEC_ECANCELED while the rest complete; timed waits return instead of hanging. No test
here faults, traps or hangs a GPU."""
import numpy as np
import pytest

import paper_2108_12550_gb300 as pkg
from paper_2108_12550_gb300 import inputs as I

torch = pytest.importorskip("torch")


def test_hooks_validate_arguments_on_the_host():
    lib = pkg.load_library()
    assert lib.rmdec_debug_fail_device_allocs(-1) == pkg.EINVAL
    assert lib.rmdec_debug_fail_device_allocs(0) == pkg.OK
    slib = pkg._load_server_api(lib)
    assert slib.rmdec_server_cancel(None, 1) == pkg.EINVAL


@pytest.fixture
def disarm():
    yield
    pkg.debug_fail_device_allocs(0)


@pytest.mark.gpu
def test_injected_allocation_failures_are_reported_and_recoverable(disarm):
    m, r, P, L = 7, 2, 8, 4
    fr = I.make_frames(m, r, 300, 2.5, seed=31)
    x = torch.from_numpy(fr["llr"].astype(np.float32))
    dec = pkg.Decoder(m, r, P, L, perm_seed=5)
    # device tables are built on the first decode: its allocation fails, then succeeds
    pkg.debug_fail_device_allocs(1)
    with pytest.raises(pkg.RmdecError) as ei:
        dec.decode(x.cuda())
    assert ei.value.status == pkg.ENOMEM
    ref = dec.decode(x.cuda()).cpu()
    assert torch.equal(ref, pkg.Decoder(m, r, P, L, perm_seed=5).decode(x.cuda()).cpu())
    # host-to-host staging, graphs, autotuning and server arenas report ENOMEM too
    out = torch.zeros((300, dec.kw), dtype=torch.int32)
    pkg.debug_fail_device_allocs(1)
    with pytest.raises(pkg.RmdecError) as ei:
        dec.decode_host(x, out)
    assert ei.value.status == pkg.ENOMEM
    dec.decode_host(x, out)
    assert torch.equal(out, ref)
    pkg.debug_fail_device_allocs(1)
    with pytest.raises(pkg.RmdecError) as ei:
        dec.graph(x.pin_memory(), out.pin_memory())
    assert ei.value.status == pkg.ENOMEM
    pkg.debug_fail_device_allocs(1)
    with pytest.raises(pkg.RmdecError) as ei:
        dec.autotune(n_frames=512)
    assert ei.value.status == pkg.ENOMEM
    pkg.debug_fail_device_allocs(1)
    with pytest.raises(pkg.RmdecError) as ei:
        pkg.Server(n_streams=1, arena_bytes=1 << 20)
    assert ei.value.status == pkg.ENOMEM
    srv = pkg.Server(n_streams=1, arena_bytes=1 << 20)
    srv.close()
    assert torch.equal(dec.decode(x.cuda()).cpu(), ref)


@pytest.mark.gpu
def test_cancel_before_admission():
    big_dec = pkg.Decoder(9, 2, 20, 4, perm_seed=1)
    small = pkg.Decoder(7, 2, 8, 4, perm_seed=2, dtype="i8")
    srv = pkg.Server(n_streams=1, arena_bytes=256 << 20, max_batch_frames=1 << 16)
    cb, cs = srv.add_decoder(big_dec), srv.add_decoder(small)
    fb = I.make_frames(9, 2, 4096, 2.5, seed=3)
    xb = torch.from_numpy(np.tile(fb["llr"].astype(np.float32), (16, 1))).pin_memory()  # 65,536 frames
    ob = torch.zeros((xb.shape[0], big_dec.kw), dtype=torch.int32).pin_memory()
    reqs = []
    for q in range(6):
        f = I.make_frames(7, 2, 50, 2.5, seed=40 + q)
        x = torch.from_numpy(I.quantize_i8(f["llr"])).pin_memory()
        o = torch.full((50, small.kw), -1, dtype=torch.int32).pin_memory()
        reqs.append((x, o))
    rb = srv.submit(cb, xb, ob)  # occupies the only stream for milliseconds
    rids = [srv.submit(cs, x, o) for x, o in reqs]
    cancelled = [srv.cancel(rid) for rid in rids[::2]]
    for rid, ok in zip(rids[::2], cancelled):
        st, _ = srv.poll(rid, timeout_us=30_000_000)
        assert st == (pkg.ECANCELED if ok else pkg.OK)
    assert any(cancelled)  # the stream was busy, so these were still queued
    alone = pkg.Decoder(7, 2, 8, 4, perm_seed=2, dtype="i8")  # the server's handles stay its own
    for (x, o), rid in zip(reqs[1::2], rids[1::2]):
        assert srv.poll(rid, timeout_us=30_000_000)[0] == pkg.OK
        assert torch.equal(o, alone.decode(x.cuda()).cpu())
    for (x, o), ok in zip(reqs[::2], cancelled):
        if ok:
            assert torch.all(o == -1)  # a cancelled request never touches its buffers
    assert srv.poll(rb, timeout_us=60_000_000)[0] == pkg.OK
    with pytest.raises(pkg.RmdecError):
        srv.cancel(rb)  # retired: unknown id
    s = srv.stats()
    assert s["cancelled"] == sum(cancelled) and s["queued"] == 0
    srv.close()


@pytest.mark.gpu
def test_fer_sweep_resumes_from_its_checkpoint(tmp_path):
    """A sweep stopped after some chunks and restarted from its checkpoint reports the same
    totals as an uninterrupted one (every chunk draws its frames from its own seed)."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    ck = str(tmp_path / "sweep.jsonl")
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--workload", "fer_sweep", "--ebn0", "1.5",
           "--sweep-frames", "600000", "--ssc-frames", "100000", "--checkpoint", ck]

    def run():
        res = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=root)
        assert res.returncode == 0, res.stderr[-2000:]
        return json.loads(res.stdout.strip().splitlines()[-1])["points"][0]

    full = run()
    lines = open(ck).read().splitlines()
    assert len(lines) == 3  # chunks of 2^18 frames
    open(ck, "w").write(lines[0] + "\n")  # as if stopped after the first chunk
    resumed = run()
    assert len(open(ck).read().splitlines()) == 3
    for name in ("p-FHT-FSCL-4-20", "p-FHT-FSCL-4-20 FP16 LLRs", "p-FHT-FSCL-4-20 INT8 LLRs", "Aut-SSC-512"):
        assert resumed[name]["errors"] == full[name]["errors"] and resumed[name]["frames"] == full[name]["frames"]
    assert full["p-FHT-FSCL-4-20"]["errors"] > 0
