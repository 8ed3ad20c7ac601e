"""Write tests/golden/config1_oracle_100steps.npz with the CPU oracle only.

Config: N = 24, 32 Coulomb factors, seed 0, dt = 0.02, the pulse
E(t) = 0.1 sin^2(pi t/10) sin t, 100 Heun steps of Eq. (equalt) with the GKBA
second-Born collision integral (oracle.propagate, with the paper's Eq. (2b-opt)
contraction route).  Stored every 10 steps:
rho(t_n), I(t_n), and at every step Tr rho and the energies.
Run: python tests/golden/make_config1_oracle.py   (about ten minutes on CPU)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gkba_inputs as gi  # noqa: E402
import oracle as O  # noqa: E402


def main():
    N, nP, dt, n = 24, 32, 0.02, 100
    s = gi.system(N, nP, seed=0)
    E = gi.field(dt * np.arange(n + 1))
    p = O.propagate(s["h"], s["v"], s["d"], s["rho0"], dt, n, E, route="paper")
    idx = np.arange(0, n + 1, 10)
    np.savez_compressed(os.path.join(HERE, "config1_oracle_100steps.npz"),
                        steps=idx, rho=p.rho[idx], I=p.I[idx],
                        trace=np.trace(p.rho, axis1=1, axis2=2).real,
                        energy_total=p.energy_total, energy_corr=p.energy_corr,
                        N=N, nP=nP, dt=dt, seed=0)


if __name__ == "__main__":
    main()
