"""Physics checks of the paper's flat-band application on the GPU path.

The BCL chain (t1 = t4 = -0.2, t2 = t3 = 1) at half filling of its flat
band (N_up = N_dn = cells / 2) is a ferromagnet in its ground state (SM Sec.
IV).  In the S^z_tot = 0 sector the A1-sublattice S^zz(q=0) tends to 1/16 as
T -> 0 (SM Eq. S33), and S^z_tot = 0 makes S^zz_11 + S^zz_22 + 2 S^zz_12
vanish in every measurement."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as p

    p.load()
    return p


def test_flatband_low_temperature_limits(lq):
    from paper_2601_08552_gb300 import physics

    rows = physics.flatband_ferro(cells=16, betas=(1.0, 16.0), U=2.0, chains=64, warm=50, sweeps=150)
    hot, cold = rows
    for r in rows:
        assert r["sum_rule_max_abs"] < 1e-9
        assert abs(r["szz_11"] - r["szz_00"]) < 1e-9 and abs(r["szz_01"] + r["szz_00"]) < 1e-9
    assert abs(cold["szz_00"] - 1.0 / 16.0) < 5.0 * cold["szz_00_err"] + 2e-4
    assert cold["s_par"] > hot["s_par"] + 0.1
