"""Writes tests/golden/full_horizon.json: the FP64 oracle's results for the transmon
pair (D = 16, N = 10^4 steps of 0.005 ns) and the fluxonium cross-resonance pair
(D = 25, N = 10^4 steps of 0.01 ns) over their whole horizons, and two columns of
the 6-fluxonium chain (D = 4096, N = 6000 steps of 0.01 ns) by the matrix-free
evolution, for the GPU accuracy tests at the step counts these workloads run.

The target of each is the unitary polar factor of the oracle's own computational
block (so F is close to 1 and a difference of 1e-5 in F is a difference in
infidelity); the stored values are F_avg, F_state, the block U_c and the exact
discrete-adjoint gradient of F_avg for every parameter (pulse, E_J/E_C/E_L per
mode, J per coupling; Sec. 2.5).  Only the oracle computes them; the workload
module supplies the seeded parameter draws.

    python tests/golden/make_full_horizon.py      # ~5 minutes on one core
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.evolve import (adjoint_gradient, comp_map, evolve_and_fidelity,  # noqa: E402
                           frame_epilogue, initial_columns, rk4_evolve_matrix_free)
from oracle.system import OracleSystem                           # noqa: E402
from paper_2406_18155_gb300 import workloads as W                # noqa: E402

CASES = {
    "transmon_pair": lambda: W.transmon_pair(seed=0),
    "fluxonium_pair_cr": lambda: W.fluxonium_pair_cr(seed=0),
}


def polar(U):
    u, _, vh = np.linalg.svd(U)
    return u @ vh


def pairs(a):
    a = np.asarray(a, dtype=np.complex128)
    return np.stack([a.real, a.imag], axis=-1).tolist()


def main():
    out = {"source": "FP64 oracle (dense Kronecker H(t), RK4, Eq. D2 fidelity, discrete adjoint) "
                     "written by tests/golden/make_full_horizon.py",
           "cases": {}}
    for name, make in CASES.items():
        wl = make()
        r = evolve_and_fidelity(wl)
        # D_c x D_c block: the evolved computational columns placed at their labels
        _, cols = comp_map(r["sys"])
        U = np.zeros((r["Uc"].shape[0],) * 2, dtype=np.complex128)
        for s, j in enumerate(cols):
            if j >= 0:
                U[:, j] = r["Uc"][:, s]
        target = polar(U)
        wl["target"] = target
        r = evolve_and_fidelity(wl)
        F, g, prms = adjoint_gradient(wl, kind="avg")
        out["cases"][name] = {"seed": 0, "N": r["sys"].N, "dt": wl["dt"], "T": wl["T"],
                              "target": pairs(target), "Uc": pairs(r["Uc"]),
                              "F_avg": r["F_avg"], "F_state": r["F_state"],
                              "grad_avg": list(map(float, g)),
                              "params": [list(map(str, p)) for p in prms]}
        print(name, r["F_avg"], r["F_state"], flush=True)
    # 6-fluxonium chain: two columns, matrix-free, whole horizon; the 64 computational
    # rows and 64 seeded other rows of each, and the column norms
    wl = W.fluxonium_chain6(seed=0)
    cols = [wl["col_index"][0], wl["col_index"][37]]
    sysm = OracleSystem(wl)
    psi = frame_epilogue(sysm, rk4_evolve_matrix_free(sysm, initial_columns(sysm, cols)))
    comp = W.comp_states([4] * 6)
    rng = np.random.Generator(np.random.PCG64(11))
    other = sorted(set(int(r) for r in rng.choice(sysm.D, size=80, replace=False)) - set(comp))[:64]
    rows = list(comp) + other
    out["cases"]["fluxonium_chain6"] = {"seed": 0, "N": sysm.N, "col_index": [int(c) for c in cols],
                                        "rows": rows, "psi_rows": pairs(psi[rows, :]),
                                        "norms": list(map(float, np.linalg.norm(psi, axis=0)))}
    print("fluxonium_chain6", np.linalg.norm(psi, axis=0), flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_horizon.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
