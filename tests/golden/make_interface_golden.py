"""Write tests/golden/interface_64x64x192.json from the oracle alone.

The 64x64x192 interface (20 x 20 x 60 bohr, a deep dense slab of Gaussian
wells against a shallow sparse one, 512 occupied states, 49 095 plane waves)
stands in for the paper's 1560-electron interface (Sec. IV).  Its dense H
(49 095^2) and dense chi0bar do not fit, so the oracle's large-system routes
(oracle/iterative.py) compute, with no input from the CUDA library:

* the 513 lowest Kohn-Sham eigenvalues (Lanczos on the grid-applied H);
* for 8 seeded perturbing potentials dV_j (sums of periodic Gaussians) and
  a spread of occupied states v (HOMO included, none closer than 1e-4 Ha to
  a neighbour, so that psi_v is unique up to sign), the Sternheimer
  solution P_c dpsi_vj of Eq. stern by preconditioned CG to 1e-12: its norm,
  the second-order energy <dV_j psi_v | dpsi_vj> (independent of the sign
  of psi_v), and its 16 largest components together with the 16 largest
  components of psi_v (which fix the sign);
* chi0bar phi for 2 seeded unit PDEP vectors (Eqs. stern, deltani,
  chiisamatrixinpdep, all 512 occupied states): phi_i^T chi0bar phi_j, the
  norms, the 64 largest components, and dn(r) at its 64 largest points.

Run:  python tests/golden/make_interface_golden.py [--states-cache FILE.npz]
(about 1-2 h on 8 cores; the cache keeps the eigenpairs between runs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402
from oracle import iterative as it  # noqa: E402
from oracle.basis import Basis  # noqa: E402
from oracle.hamiltonian import KSStates  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "interface_64x64x192.json")
PERT_SEED = 1501031440
PHI_SEED = 1501031441
N_PERT = 8
N_PHI = 2
TARGET_STATES = (0, 102, 204, 306, 408, 511)


def pick_states(eps, n_occ, targets, min_sep=1e-4):
    """Nearest occupied index to each target whose neighbours are >= min_sep away."""
    ok = []
    for v in range(n_occ):
        lo = eps[v] - eps[v - 1] if v > 0 else np.inf
        hi = eps[v + 1] - eps[v]
        if lo >= min_sep and hi >= min_sep:
            ok.append(v)
    ok = np.asarray(ok)
    out = []
    for t in targets:
        v = int(ok[np.argmin(np.abs(ok - t))])
        if v not in out:
            out.append(v)
    return out


def top(x, k):
    idx = np.argsort(-np.abs(x))[:k]
    idx = np.sort(idx)
    return idx.tolist(), x[idx].tolist()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--states-cache", default=None)
    args = ap.parse_args()
    s = synthetic.make_system("interface")
    b = Basis(s.grid, s.cell)
    t0 = time.time()
    if args.states_cache and os.path.exists(args.states_cache):
        z = np.load(args.states_cache)
        ks = KSStates(eps=z["eps"], C=z["C"], n_occ=s.n_occ)
    else:
        ks = it.ks_states_lanczos(b, s.v_r, s.n_occ, n_states=s.n_occ + 1, tol=1e-14)
        if args.states_cache:
            np.savez(args.states_cache, eps=ks.eps, C=ks.C)
    print(f"states: {time.time() - t0:.0f} s, gap {ks.gap:.6f} Ha", flush=True)
    res = it.apply_h(b, s.v_r, ks.C.T) - ks.eps[:, None] * ks.C.T
    state_res = float(np.linalg.norm(res, axis=1).max())
    print(f"largest eigen-residual {state_res:.2e}", flush=True)
    del res
    states = pick_states(ks.eps, s.n_occ, TARGET_STATES)
    u_occ = it.to_grid(b, ks.C[:, : s.n_occ].T)
    dvs = synthetic.random_grid_potentials(PERT_SEED, N_PERT, s.grid, s.cell)
    items = []
    for j in range(N_PERT):
        t1 = time.time()
        dpsi, its, rres = it.sternheimer_pcg(b, ks, s.v_r, dvs[j], states=states, tol=1e-12,
                                             u_occ=u_occ)
        w = it.from_grid(b, dvs[j][None] * u_occ[states])
        for k, v in enumerate(states):
            x = dpsi[v]
            pi, pv = top(ks.C[:, v], 16)
            di, dvv = top(x, 16)
            items.append({"j": j, "v": v, "dpsi_norm": float(np.linalg.norm(x)),
                          "e2": float(w[k] @ x), "psi_idx": pi, "psi_val": pv,
                          "dpsi_idx": di, "dpsi_val": dvv, "iters": int(its[k]),
                          "residual": float(rres[k])})
        print(f"perturbation {j}: {time.time() - t1:.0f} s, iters {its.tolist()}", flush=True)
    phi = synthetic.random_vectors(PHI_SEED, N_PHI, b.n_pdep_dim)
    phi /= np.linalg.norm(phi, axis=1)[:, None]
    t1 = time.time()
    chi, dn = it.chi0bar_apply_pcg(b, ks, s.v_r, phi, tol=1e-12, return_dn=True)
    print(f"chi0bar on {N_PHI} vectors: {time.time() - t1:.0f} s", flush=True)
    chi0 = {"seed": PHI_SEED, "n": N_PHI, "tol": 1e-12, "M": (phi @ chi.T).tolist(),
            "norm": np.linalg.norm(chi, axis=1).tolist(), "idx": [], "val": [],
            "dn_idx": [], "dn_val": [], "dn_max": []}
    for j in range(N_PHI):
        i, v = top(chi[j], 64)
        chi0["idx"].append(i)
        chi0["val"].append(v)
        d = dn[j].ravel()
        i, v = top(d, 64)
        chi0["dn_idx"].append(i)
        chi0["dn_val"].append(v)
        chi0["dn_max"].append(float(np.abs(d).max()))
    out = {"what": "oracle reference values for the 64x64x192 interface workload "
                   "(written by tests/golden/make_interface_golden.py from oracle/ alone)",
           "system": "interface", "grid": list(s.grid), "cell": list(s.cell), "n_pw": b.n_pw,
           "n_occ": s.n_occ, "eps": ks.eps.tolist(), "max_eigen_residual": state_res,
           "perturbations": {"seed": PERT_SEED, "n": N_PERT, "states": states, "tol": 1e-12,
                             "items": items},
           "chi0": chi0}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
