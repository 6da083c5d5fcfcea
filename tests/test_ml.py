"""RM(2,5) with P = 4, L = 2 at 3 dB, 10^4 frames (the small configuration): the GPU decoder's
word against brute-force maximum likelihood over all 2^16 codewords. On these frames the
decoder finds the ML word every time (checked on the oracle as well); a different word is
accepted only at an exact correlation tie."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402


def test_gpu_decoder_finds_the_ml_codeword_on_rm25():
    m, r, P, L = 5, 2, 4, 2
    n, k = I.rm_dims(m, r)
    fr = I.make_frames(m, r, 10000, 3.0, seed=2021)
    llr = fr["llr"].astype(np.float32)
    # brute force: the codeword of largest correlation sum_i (1 - 2 x_i) llr_i
    U = ((np.arange(1 << k)[:, None] >> np.arange(k)) & 1).astype(np.uint8)
    S = (1.0 - 2.0 * I.encode(U, m, r)).astype(np.float64)
    corr_ml = np.empty(len(llr))
    ml_info = np.empty((len(llr), k), dtype=np.uint8)
    for c0 in range(0, len(llr), 1000):
        c = llr[c0:c0 + 1000].astype(np.float64) @ S.T
        b = np.argmax(c, axis=1)
        ml_info[c0:c0 + 1000] = U[b]
        corr_ml[c0:c0 + 1000] = c[np.arange(len(b)), b]
    dec = pkg.Decoder(m, r, P, L, perm_seed=1)
    out = dec.decode(torch.from_numpy(llr).cuda()).cpu().numpy()
    info = pkg.unpack_bits(out, k)
    diff = np.any(info != ml_info, axis=1)
    corr_gpu = np.sum((1.0 - 2.0 * I.encode(info, m, r)) * llr.astype(np.float64), axis=1)
    assert np.all(corr_gpu <= corr_ml + 1e-9)  # ML is optimal
    assert np.all(np.abs(corr_gpu[diff] - corr_ml[diff]) <= 1e-6 * np.abs(corr_ml[diff])), diff.sum()
    assert diff.mean() <= 1e-3
    fer_gpu = np.mean(np.any(info != fr["u"], axis=1))
    fer_ml = np.mean(np.any(ml_info != fr["u"], axis=1))
    print(f"RM(2,5) P=4 L=2 3 dB: GPU = ML on {1 - diff.mean():.4%} of frames; FER {fer_gpu:.4f} (ML {fer_ml:.4f})")
