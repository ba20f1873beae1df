"""Write synthetic/data/inputs.npz: element maps and matched Twiss parameters.

Oracle script (calls only oracle/ and the seeded-input module synthetic/).
Run:  python -m oracle.gen_inputs

Contents
  <key>.order/.C/.R/.T/.U   transport maps (orders 2 and 3) of
        D1.0  exact drift, 1.0 m
        QF    thick quadrupole L = 0.2 m, K1 = +1.2 m^-2
        QD    thick quadrupole L = 0.2 m, K1 = -1.2 m^-2
        c5.<v>.QF / c5.<v>.QD   the 64 DA-variant quadrupoles (K1 +-2 %)
  twiss.<cfg>  (beta_x, alpha_x, beta_y, alpha_y) at the lattice entrance
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synthetic as syn  # noqa: E402
from oracle import flows, maps  # noqa: E402


def main():
    out = {}

    def put(key, m):
        for f in ("C", "R", "T", "U"):
            out["%s.%s" % (key, f)] = m[f]
        out[key + ".order"] = np.array(m["order"])

    for order in (2, 3):
        put("D1.0.o%d" % order, maps.drift_map(syn.L_DRIFT, order))
        put("QF.o%d" % order, maps.quad_map(syn.L_QUAD, syn.K1_QUAD, order))
        put("QD.o%d" % order, maps.quad_map(syn.L_QUAD, -syn.K1_QUAD, order))
    params = syn.c5_params()
    for v in range(params.shape[0]):
        kf, kd = syn.c5_strengths(params[v])[:2]
        put("c5.%d.QF" % v, maps.quad_map(syn.L_QUAD, kf, 2))
        put("c5.%d.QD" % v, maps.quad_map(syn.L_QUAD, kd, 2))

    R = {k: out[k + ".R"] for k in ("D1.0.o2", "QF.o2", "QD.o2")}
    c1 = maps.compose_linear([R["QF.o2"], R["D1.0.o2"], R["QD.o2"], R["D1.0.o2"]])
    c3 = maps.compose_linear([R["D1.0.o2"], R["QF.o2"], R["D1.0.o2"], R["QD.o2"]])
    cell2 = syn.lattice_c2(cells=1, rf=False)["elements"]

    def c2_flow(z):
        for e in cell2:
            if e["type"] in ("KQUAD", "KSEXT"):
                z = flows.thick_multipole(z, e["L"], e.get("K1", 0.0), e.get("K2", 0.0), e["n_kicks"])
            else:
                z = flows.exact_drift(z, e["L"])
        return z

    c2 = maps.jacobian(c2_flow)
    for name, M in (("c1", c1), ("c2", c2), ("c3", c3)):
        (bx, ax), (by, ay) = maps.twiss_from_cell(M)
        out["twiss." + name] = np.array([bx, ax, by, ay])
    os.makedirs(os.path.dirname(syn.DATA), exist_ok=True)
    np.savez_compressed(syn.DATA, **out)
    print("wrote", syn.DATA, len(out), "arrays")


if __name__ == "__main__":
    main()
