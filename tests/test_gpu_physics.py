"""Physics sanity, independent of the oracle: a Neo-Hookean block resting on
the sticky floor under gravity shortens less the stiffer it is, and its
shortening follows the linear-elastic scale rho g H^2 / (2 E) of a column
compressed by its own weight.  The block's height is measured between its top
and bottom layers, which leaves out the part-cell sinking of the bottom into
the sticky floor band; the time average over the free oscillation, which the
undamped method does not dissipate, is the static value."""
import numpy as np
import pytest

from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def test_gravity_sag_scales_with_inverse_stiffness(M):
    n = 32
    x = scenes.jittered_lattice((10, 3, 10), (22, 11, 22), n, (2, 2, 2), seed=3)   # 12 x 8 x 12 cells
    H = 8.0 / n
    top = x[:, 1] > np.quantile(x[:, 1], 0.95)
    bottom = x[:, 1] < np.quantile(x[:, 1], 0.05)
    sags = {}
    for E in (2e4, 4e4, 8e4):
        sc = scenes.Scene("sag", n_grid=n, dt=1e-4, E=E, nu=0.3, rho=1e3, x=x, particle_volume=(1.0 / n) ** 3 / 8)
        sim = M.sim_from_scene(sc)
        h0 = float(x[top, 1].mean() - x[bottom, 1].mean())
        hs = []
        for call in range(40):                       # 1 s of simulated time
            sim.step(250)
            if call >= 10:
                y = sim.read()["x"][:, 1]
                hs.append(float(y[top].mean() - y[bottom].mean()))
        sim.close()
        sags[E] = h0 - np.mean(hs)
    s = [sags[E] for E in sorted(sags)]
    assert s[0] > s[1] > s[2] > 0, sags
    # shortening ~ 1 / E at small strain (at E = 1e4, 2% strain, the Neo-Hookean
    # volume term already stiffens the column by about 20 %)
    scaled = [sags[E] * E for E in sorted(sags)]
    assert max(scaled) / min(scaled) < 1.15, scaled
    lin = 1e3 * 9.8 * H ** 2 / 2.0                      # 1-D self-weight shortening x E
    assert abs(scaled[-1] / lin - 1.0) < 0.15, (scaled, lin)
