"""Frame error rates of the long-list and RM(4, m) decoders against the values the paper
prints (Fig. 4), on the GPU: frames generated on the device from a seeded generator, about 60
expected errors per point, and the same factor-2.2 band as the oracle's FER pins (wide enough
for the sample and the unstated Eb/N0 convention, narrow enough to catch a wrong list rule).
The decoders are bit-exact against the integer oracle on small frame counts
(test_gpu_parity.py); this checks them at the paper's operating points."""
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_12550_gb300 as pkg  # noqa: E402
from paper_2108_12550_gb300 import inputs as I  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_fer_long_lists.txt")


def _rows():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            t = line.split()
            rows.append((int(t[0]), int(t[1]), t[2], int(t[3]), int(t[4]), float(t[5]), float(t[6]), " ".join(t[7:])))
    return rows


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[7].replace(" ", "_") + f"@{r[5]}dB")
def test_fer_matches_paper_figure(row):
    m, r, dec_kind, P, L, eb, fer_paper, _ = row
    n = int(min(1 << 18, max(1 << 13, 60 / fer_paper)))
    k = I.rm_dims(m, r)[1]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4100 + m * 100 + r * 10 + L)
    u, llr = I.make_frames_torch(m, r, n, eb, gen)
    if dec_kind == "pfht":
        dec = pkg.Decoder(m, r, P, L, perm_seed=7)
    else:
        dec = pkg.Decoder(m, r, 1, L, algo="fhtfscl")
    words = dec.decode(llr.contiguous())
    kw = (k + 31) // 32
    got = ((words.view(-1, kw, 1) >> torch.arange(32, device="cuda")) & 1).view(-1, 32 * kw)[:, :k]
    fer = torch.any(got.to(torch.uint8) != u, dim=1).sum().item() / n
    print(f"{row[7]} at {eb} dB: FER {fer:.3g} over {n} frames (paper {fer_paper:.3g})")
    assert fer_paper / 2.2 <= fer <= fer_paper * 2.2, (fer, n, fer_paper)
