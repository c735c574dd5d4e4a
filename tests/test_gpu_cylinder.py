"""Flow past a cylinder with droplets (the paper's Sec. 5 case) on the periodic
two-way carrier, at half resolution (128^2, R = 6.4 cells).  The paper gives
figures only, so these are physical and statistical checks, not parity: the
clean flow's drag is that of a confined cylinder at Re = 20, the FLA-coupled
and PSI-CELL-coupled runs give correlated momentum-source profiles where the
droplets have arrived, and the droplets change the drag."""
import numpy as np
import pytest

from paper_2512_20829_gb300 import cylinder as CY
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def test_cylinder_re20_fla_against_psicell(ctx):
    case = I.cylinder_flow(re=20.0, scale=2, nsteps=600, warm_steps=800)
    fl = CY.run(ctx, case, "fla")
    ps = CY.run(ctx, case, "psicell")
    off = CY.run(ctx, case, "fla", coupled=False)
    cmp = CY.compare(fl, ps)
    print(f"\nRe 20, 128^2: C_d clean {fl['cd_clean']:.3f}; end of run C_d FLA {fl['cd'][-1]:.4f} "
          f"PSI-CELL {ps['cd'][-1]:.4f} uncoupled {off['cd'][-1]:.4f}")
    for st, c in cmp.items():
        print(f"  x/R = {st:2d}: S_mom_y profile correlation {c['corr']:.3f}, norm ratio FLA/PSI-CELL "
              f"{c['norm_ratio']:.3f}")
    # a confined cylinder (R/L = 0.05 blockage in a periodic box, penalised) at Re = 20
    # has a drag coefficient of order 2-5 (2 for an unbounded one)
    assert 1.0 < fl["cd_clean"] < 8.0
    assert abs(fl["cl_clean"]) < 0.05 * fl["cd_clean"]                  # steady, near-symmetric wake
    # the droplets add drag on the carrier that the uncoupled run does not see
    assert abs(fl["cd"][-1] - off["cd"][-1]) > 1e-4 * abs(off["cd"][-1])
    # where the droplets have arrived by t = 0.6 (x/R = 0, 3) the two coupled runs'
    # momentum-source profiles agree in shape
    for st in (0, 3):
        assert cmp[st]["corr"] > 0.5
    assert np.all(np.isfinite(fl["S_mom_y"])) and np.all(np.isfinite(ps["S_mom_y"]))
