"""Decision-mismatch rates of the input precisions against the FP64 oracle.

The same seeded frames at the operating points are decoded by the GPU from FP32, FP16 and
INT8 (step 0.25, saturated at +-127) LLRs and by the FP64 oracle from the exact channel
LLRs, and by the tensor-core Hadamard variant from FP16 LLRs. FP32 decides like FP64 except at
near-ties; the quantised inputs change the metric
itself, so their words may differ wherever the quantisation moves a decision.

The bounds follow the measured rates. On these seeded frames every input type decides every
frame as the FP64 oracle does; the long FER sweeps put the rates against FP32 at about 1e-6
(FP16) and 5e-5 (INT8, RM(2,9) at 2.25 dB), i.e. an expected 0.003 and 0.15 differing frames
here. A bound of two frames is therefore far above the expected count (a Poisson count of mean
0.15 reaches 3 with probability 5e-4) and far below what a broken widening or quantiser
produces (hundreds of frames).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402

# (m, r, P, L, Eb/N0, frames, largest tolerated number of frames decided unlike FP64)
POINTS = [
    (9, 2, 20, 4, 2.25, 3000, {"f32": 2, "f16": 2, "i8": 2, "f16_tensor_hadamard": 2}),
    (9, 3, 16, 8, 4.0, 600, {"f32": 2, "f16": 2, "i8": 2, "f16_tensor_hadamard": 2}),
]


@pytest.mark.parametrize("m,r,P,L,eb,nf,bound", POINTS, ids=["rm29_p20_l4", "rm39_p16_l8"])
def test_mismatch_rates_vs_fp64_oracle(m, r, P, L, eb, nf, bound):
    fr = I.make_frames(m, r, nf, eb, seed=4242)
    perms = I.perm_table(m, r, P, L, seed=1)
    ref = O.decode(m, r, P, L, perms, fr["llr"])
    inputs = {"f32": fr["llr"].astype(np.float32), "f16": I.to_f16(fr["llr"]), "i8": I.quantize_i8(fr["llr"]),
              "f16_tensor_hadamard": I.to_f16(fr["llr"])}
    rates = {}
    for dt, x in inputs.items():
        dec = pkg.Decoder(m, r, P, L, dtype=dt[:3], perms=perms)
        if dt.endswith("tensor_hadamard"):
            dec.set_hadamard("tensor")
        out = dec.decode(torch.from_numpy(x).cuda()).cpu().numpy()
        info = pkg.unpack_bits(out, dec.k)
        rates[dt] = float(np.mean(np.any(info != ref["info"], axis=1)))
        fer = float(np.mean(np.any(info != fr["u"], axis=1)))
        print(f"RM({r},{m}) P={P} L={L} {eb} dB {dt}: decisions differing from FP64 {rates[dt]:.4%} "
              f"(FER {fer:.4%}, FP64 oracle FER {np.mean(np.any(ref['info'] != fr['u'], axis=1)):.4%})")
    for dt, b in bound.items():
        assert rates[dt] * nf <= b, (dt, rates[dt] * nf)
