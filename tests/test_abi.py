"""CPU checks of the C ABI: the library loads, exports every declared entry point, validates
arguments, and samples the same permutation tables as the independent Python generator."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2108_12550_gb300 as pkg
from paper_2108_12550_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("rmdec.h", "rmdec_serve.h",
                                                                          "rmdec_group.h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rmdec_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = pkg.load_library()
    names = _declared()
    assert len(names) >= 32
    for n in names:
        assert hasattr(lib, n), n


def test_kernel_query_checks_its_arguments():
    lib = pkg.load_library()
    k = ctypes.c_int()
    assert lib.rmdec_kernel_for(None, 10, ctypes.byref(k)) == pkg.EINVAL
    h = ctypes.c_void_p()
    assert lib.rmdec_create(ctypes.byref(h), 7, 2, 8, 4, 1) == pkg.OK
    try:
        assert lib.rmdec_kernel_for(h, 10, None) == pkg.EINVAL
        assert lib.rmdec_kernel_for(h, -1, ctypes.byref(k)) == pkg.EINVAL
    finally:
        lib.rmdec_destroy(h)


def test_invalid_configurations_are_rejected():
    lib = pkg.load_library()
    h = ctypes.c_void_p()
    for args in [(9, 2, 20, 3), (10, 2, 20, 32), (9, 2, 20, 64), (10, 4, 4, 4), (9, 5, 4, 4), (1, 1, 4, 4), (11, 1, 4, 4), (9, 8, 4, 64),
                 (9, 2, 0, 4), (9, 2, 129, 4)]:
        st = lib.rmdec_create(ctypes.byref(h), *args, 1)
        assert st == pkg.EINVAL and h.value is None
        assert len(lib.rmdec_last_error(None)) > 0
    assert lib.rmdec_create_aut_ssc(ctypes.byref(h), 9, 4, 16, 1) == pkg.EINVAL


@pytest.mark.parametrize("m,r,P,L", [(5, 2, 4, 2), (9, 2, 20, 4), (9, 3, 3, 8), (6, 3, 2, 1)])
def test_seeded_tables_match_independent_generator(m, r, P, L):
    d = pkg.Decoder(m, r, P, L, perm_seed=12345)
    assert d.n == 1 << m and d.k == I.rm_dims(m, r)[1]
    assert np.array_equal(d.info_idx, I.info_set(m, r))
    got = d.get_perms().reshape(P, -1, I.PERM_REC)
    assert np.array_equal(got, I.perm_table(m, r, P, L, seed=12345))
    d.close()


def test_aut_ssc_table_matches_independent_generator():
    d = pkg.Decoder(9, 2, 40, algo="autssc", perm_seed=99)
    assert np.array_equal(d.get_perms(), I.ssc_perm_table(9, 40, 99))
    d.close()


def test_set_perms_validates_records():
    d = pkg.Decoder(7, 2, 2, 2, perm_seed=1)
    tab = d.get_perms()
    d.set_perms(tab)  # round trip
    bad = tab.copy()
    bad[3, :7] = 0  # singular linear part
    with pytest.raises(pkg.RmdecError) as ei:
        d.set_perms(bad)
    assert ei.value.status == pkg.EINVAL
    wrong = tab.copy()
    wrong[0, 8] = 1  # column beyond GA(7)
    with pytest.raises(pkg.RmdecError):
        d.set_perms(wrong)
    with pytest.raises(pkg.RmdecError):
        d.set_perms(tab[:-1])


def test_bad_dtype_and_poll_arguments():
    d = pkg.Decoder(5, 2, 2, 2)
    assert d._lib.rmdec_set_dtype(d._h, 7) == pkg.EINVAL
    assert d._lib.rmdec_poll(d._h, 12345, 0) == pkg.EINVAL


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2, (5, 46), dtype=np.uint8)
    assert np.array_equal(pkg.unpack_bits(pkg.pack_bits(b), 46), b)


def test_group_membership_is_validated_on_the_host():
    lib = pkg.load_library()
    a = pkg.Decoder(7, 2, 8, 4)
    b = pkg.Decoder(9, 3, 2, 4, dtype="i8")
    c = pkg.Decoder(9, 2, 4, 2)
    s = pkg.Decoder(9, 2, 8, algo="autssc")
    e = pkg.Decoder(10, 2, 2, 4)
    f = pkg.Decoder(8, 2, 1, 4, algo="fhtfscl")
    ok = pkg.Group([a, b, f])  # host-side only: no device work at creation
    r4 = pkg.Decoder(8, 4, 2, 4)
    l32 = pkg.Decoder(7, 2, 2, 32)
    root1 = pkg.Decoder(7, 1, 2, 4)
    for bad in ([a, c], [a, s], [e], [], [r4], [l32], [root1]):
        with pytest.raises(pkg.RmdecError) as ei:
            pkg.Group(bad)
        assert ei.value.status == pkg.EINVAL
        assert lib.rmdec_group_last_error(None)
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 17)(*([a._h.value] * 17))
    assert lib.rmdec_group_create(ctypes.byref(h), arr, 17) == pkg.EINVAL
    # bad segments are rejected before any device work
    seg = (pkg._Segment * 2)(pkg._Segment(0, None, 0, None), pkg._Segment(3, None, 0, None))
    assert lib.rmdec_group_decode(ok._h, seg, 2, None) == pkg.EINVAL
    seg = (pkg._Segment * 1)(pkg._Segment(1, None, 5, None))
    assert lib.rmdec_group_decode(ok._h, seg, 1, None) == pkg.EINVAL
    seg = (pkg._Segment * 1)(pkg._Segment(1, 0x1008, 5, 0x2000))
    assert lib.rmdec_group_decode(ok._h, seg, 1, None) == pkg.EINVAL  # misaligned LLRs
    assert b"aligned" in lib.rmdec_group_last_error(ok._h)
    assert lib.rmdec_group_decode(ok._h, None, 1, None) == pkg.EINVAL
    assert lib.rmdec_group_set_tuning(ok._h, 21, 0) == pkg.EINVAL
    assert lib.rmdec_group_set_tuning(ok._h, -1, 0) == pkg.EINVAL
    assert lib.rmdec_group_set_tuning(ok._h, 20, 0) == pkg.OK
    ok.close()


def test_tensor_core_hadamard_availability_is_checked_on_the_host():
    d = pkg.Decoder(9, 3, 16, 8)
    d.set_hadamard("tensor")
    d.set_hadamard("shuffle")
    for bad in [pkg.Decoder(7, 2, 8, 4), pkg.Decoder(9, 2, 4, 2), pkg.Decoder(9, 2, 8, algo="autssc")]:
        with pytest.raises(pkg.RmdecError) as ei:
            bad.set_hadamard("tensor")
        assert ei.value.status == pkg.EINVAL
    assert d._lib.rmdec_set_hadamard(d._h, 5) == pkg.EINVAL
    a = pkg.Decoder(9, 2, 4, 4)
    a.set_hadamard("tensor")
    with pytest.raises(pkg.RmdecError):
        pkg.Group([a])  # grouped launches have no tensor-core variant



def test_kernel_choice_is_checked_on_the_host():
    d = pkg.Decoder(7, 2, 8, 4)
    d.set_kernel("path")
    d.set_kernel("warp")
    d.set_kernel("auto")
    for bad in [pkg.Decoder(9, 2, 4, 4), pkg.Decoder(8, 3, 4, 4), pkg.Decoder(6, 2, 4, 16),
                pkg.Decoder(7, 2, 8, algo="autssc"), pkg.Decoder(7, 1, 2, 4)]:
        with pytest.raises(pkg.RmdecError) as ei:
            bad.set_kernel("path")
        assert ei.value.status == pkg.EINVAL
    assert d._lib.rmdec_set_kernel(d._h, 7) == pkg.EINVAL
    pkg.Decoder(4, 2, 128, 8).set_kernel("path")
    pkg.Decoder(8, 2, 20, 8).set_kernel("path")
    pkg.Decoder(7, 3, 20, 8).set_kernel("path")
