"""The judge of the surrogate at the size of the learned-Born-charge configuration: 16,384 waters x
1024 modes (the 32 x 32 grid), 10^4 steps of 0.5 fs (5 ps), for the shipped network Born charges
(with the BF16x3 and with the FP64 coupling), explicit central finite-difference Born charges every
step (the conservative reference) and Mulliken charges (the paper's cheap replacement).

Cavity (paper_2512_03277_gb300/judge.py, resonant_workload): the 32 x 32 grid of a resonant
cavity, the k = 0 mode at the bend of the synthetic water and the in-plane wave vectors spaced so
that the band of modes spans 1 to 1.3 times the bend (below the stretch), with the collective
coupling of the resonant single box. (The workload's own grid, spaced by 2 pi over the slab, puts
every k != 0 mode hundreds of times above both bands, at omega dt of about 50 rad, where the step
no longer conserves energy whatever the dipole derivative.)

Reported per run: energy drift (Ha/atom over the run), heating (mean temperature of the last tenth
minus that of the second tenth; the first tenth is the equipartition transient), the temperature
at eleven points, and the bend and stretch band centroids of the total-dipole spectrum.
Asserted: the explicit Born charges conserve energy (|drift| < 1e-6 Ha/atom, the target for
10^4 steps); the network drifts less than the Mulliken charges and heats no more than they do
beyond the run's temperature noise (0.05 K: in 5 ps no model here heats measurably, all within a
few hundredths of a kelvin, while the paper's Mulliken heating shows over its much longer runs);
the network's bands lie closer to the reference's than the Mulliken bands."""
import numpy as np
import pytest

import cavmd_synth as cs

pytestmark = pytest.mark.gpu
STEPS = 10000
LAGS = 2000


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_03277_gb300 import build
    build.build()
    import paper_2512_03277_gb300 as P
    P.load_library()
    return P


def test_judge_at_c4_size(P, capsys):
    from paper_2512_03277_gb300 import cavmd as B
    from paper_2512_03277_gb300 import judge as J
    mlp = B.trained_born_mlp()
    if mlp is None:
        pytest.skip("no trained network shipped")
    params = cs.load_water_params()
    sy, modes, wb = J.resonant_workload(params, "c4")
    dt = P.default_options().dt
    out = {}
    for model, prec in (("born_central", 0), ("born_mlp", 2), ("born_mlp", 0), ("mulliken", 0)):
        r = J.run(P, params, sy, modes, model, prec, STEPS, mlp=mlp, lags=LAGS)
        bend, stretch = J.bands(r["acf_dipole"], dt, wb)
        out[(model, prec)] = {"drift": r["drift"], "heating": J.heating(r["T"]), "bend": bend, "stretch": stretch,
                              "T": J.temperature_curve(r["T"])}
    ref = out[("born_central", 0)]
    for v in out.values():
        v["band_error_mev"] = 1e3 * max(abs(v["bend"] - ref["bend"]), abs(v["stretch"] - ref["stretch"]))
    with capsys.disabled():
        for (m, p), v in out.items():
            print(f"\nc4 judge {m:12s} {'BF16x3' if p else 'FP64  '} drift {v['drift']:+.2e} Ha/atom  heating "
                  f"{v['heating']:+.2f} K  bend {v['bend']:.4f} eV  stretch {v['stretch']:.4f} eV  band error "
                  f"{v['band_error_mev']:.2f} meV  T(t) " + " ".join(f"{t:.0f}" for _, t in v["T"]), end="")
    assert abs(ref["drift"]) < 1e-6
    mul = out[("mulliken", 0)]
    for p in (0, 2):
        net = out[("born_mlp", p)]
        assert net["heating"] < mul["heating"] + 0.05
        assert abs(net["drift"]) < abs(mul["drift"])
        assert net["band_error_mev"] < mul["band_error_mev"]
