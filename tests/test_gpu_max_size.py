"""CC+Euler at the size limits of the int64-offset path: a permuted grid with
more than 2^31 arcs (CSR positions past the int32 range), bit-exact against
the oracle.  Opt-in (RST_MAX_SIZE=1): it needs ~60 GB of host memory and
~110 GB of device memory, and the oracle takes minutes."""
import os

import numpy as np
import pytest

import oracle
from paper_2603_11645_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("RST_MAX_SIZE") != "1", reason="opt-in: RST_MAX_SIZE=1")]


def test_cc_euler_past_2_31_arcs():
    import paper_2603_11645_gb300 as rst
    side = 23171  # 536,895,241 vertices, 2,147,488,280 arcs > 2^31
    g = graphs.grid(side, side, seed=9, permute=True, root="random", offsets_bits=64)
    assert g.A > 2 ** 31
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    par = rst.build(off, col, g.root, "cc_euler")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rst.build(off, col, g.root, "cc_euler", out=par)
    e1.record()
    torch.cuda.synchronize()
    print(f"\nmax-size grid {side}x{side}: n={g.n} A={g.A} CC+Euler {e0.elapsed_time(e1):.1f} ms")
    got = par.cpu().numpy()
    del off, col, par
    torch.cuda.empty_cache()
    want = oracle.rst(g.n, g.offsets, g.cols, g.root)
    assert np.array_equal(got, want)
