"""Decoding without device allocation: rmdec_decode_noalloc against rmdec_decode.

Some callers may not allocate device memory when they decode: a framework whose caching
allocator owns all of the GPU's memory, a real-time loop whose memory budget is fixed at
start-up, or a plug-in inside a host process that forbids device allocations after it has
initialised. rmdec_decode_noalloc serves them: it keeps the decoder's permutation and
position tables in one fixed device array of the library instead of allocating them. Its
results must equal rmdec_decode's on the same frames, also when consecutive calls overwrite
that array with the tables of different decoders.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import paper_2108_12550_gb300 as pkg
from paper_2108_12550_gb300 import inputs as I


def _call(lib, dec, llr, out, stream):
    return lib.rmdec_decode_noalloc(dec._h, llr.data_ptr(), llr.shape[0], out.data_ptr(), stream)


def test_tables_beyond_the_fixed_array_are_rejected_before_any_device_work():
    lib = pkg.load_library()
    # RM(3,9), P = 128, L = 8: 128 decoders x 64 maps x 22 bytes, above the 128 KiB array
    big = pkg.Decoder(9, 3, 128, 8)
    st = lib.rmdec_decode_noalloc(big._h, ctypes.c_void_p(0x1000), 4, ctypes.c_void_p(0x2000), None)
    assert st == pkg.EINVAL
    assert b"fixed" in lib.rmdec_last_error(big._h)
    # zero frames: nothing to do
    assert lib.rmdec_decode_noalloc(big._h, None, 0, None, None) == pkg.OK
    big.close()


@pytest.mark.gpu
def test_noalloc_decode_equals_decode_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    lib = pkg.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    # two decoders with different tables: the headline RM(2,9) P=20 L=4 on FP32 LLRs and
    # RM(3,9) P=16 L=8 on INT8 codes; 700 and 300 frames (several waves, ragged)
    a = pkg.Decoder(9, 2, 20, 4, perm_seed=11, dtype="f32")
    b = pkg.Decoder(9, 3, 16, 8, perm_seed=12, dtype="i8")
    fa = I.make_frames(9, 2, 700, 2.25, seed=31)
    fb = I.make_frames(9, 3, 300, 3.0, seed=32)
    xa = torch.from_numpy(fa["llr"].astype(np.float32)).cuda()
    xb = torch.from_numpy(I.quantize_i8(fb["llr"])).cuda()
    ref_a = a.decode(xa)
    ref_b = b.decode(xb)
    torch.cuda.synchronize()
    out_a1 = torch.full_like(ref_a, -1)
    out_b = torch.full_like(ref_b, -1)
    out_a2 = torch.full_like(ref_a, -1)
    # two calls in a row with different tables, then the first decoder again
    assert _call(lib, a, xa, out_a1, stream) == pkg.OK, lib.rmdec_last_error(a._h)
    assert _call(lib, b, xb, out_b, stream) == pkg.OK, lib.rmdec_last_error(b._h)
    assert _call(lib, a, xa, out_a2, stream) == pkg.OK, lib.rmdec_last_error(a._h)
    torch.cuda.synchronize()
    # the same kernel on the same frames: the outputs must be identical
    assert torch.equal(out_a1, ref_a)
    assert torch.equal(out_b, ref_b)
    assert torch.equal(out_a2, ref_a)
    # and they decode the channel: the FER of these frames is small at these points
    ua = pkg.unpack_bits(out_a1.cpu().numpy(), a.k)
    assert np.mean(np.any(ua != fa["u"], axis=1)) < 0.01
    a.close()
    b.close()


@pytest.mark.gpu
def test_noalloc_decode_with_the_path_per_thread_kernel():
    # short codes decode with the path-per-thread kernel; its launch (several frames per warp)
    # reads the same fixed tables
    torch = pytest.importorskip("torch")
    lib = pkg.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    for (m, P, L, dt, nf) in [(7, 8, 4, "i8", 501), (5, 4, 2, "f32", 333), (8, 8, 4, "f32", 257)]:
        d = pkg.Decoder(m, 2, P, L, perm_seed=21, dtype=dt)
        fr = I.make_frames(m, 2, nf, 2.5, seed=40 + m)
        x = fr["llr"].astype(np.float32) if dt == "f32" else I.quantize_i8(fr["llr"])
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        ref = d.decode(xd)
        torch.cuda.synchronize()
        out = torch.full_like(ref, -1)
        assert _call(lib, d, xd, out, stream) == pkg.OK, lib.rmdec_last_error(d._h)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (m, P, L)
        d.close()
