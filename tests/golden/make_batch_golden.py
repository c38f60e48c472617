"""Write tests/golden/uneven_batch.json from the oracle alone.

The uneven batch: 32 seeded Gaussian-well systems, N in {24, 32, 40, 48, 64},
L = 10 N / 24 bohr, N_occ ~ U{8..96}, N_pdep = 2 N_occ (synthetic.make_batch).
For every member the oracle computes, with no input from the CUDA library:

* the n_occ + 1 lowest Kohn-Sham eigenvalues;
* members with N <= 32 (N_pw <= 1 935): the n_pdep most negative eigenvalues
  of the dense chi0bar by the Adler-Wiser sum over all empty states
  (Eqs. AdlerWiser, eigendecompzerofreq; oracle.pdep);
* members with N >= 40: chi0bar phi for 2 seeded unit PDEP vectors by
  Sternheimer solves over all occupied states (Eqs. stern, deltani,
  chiisamatrixinpdep; oracle.iterative, Lanczos states, CG to 1e-12):
  phi_i^T chi0bar phi_j, the norms and the 32 largest components.

Run:  python tests/golden/make_batch_golden.py   (about half an hour on 8 cores)
"""
from __future__ import annotations

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
from oracle.hamiltonian import ks_states  # noqa: E402
from oracle.pdep import chi0bar_dense, pdep_reference  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "uneven_batch.json")
PHI_SEED0 = 1501031450   # member k uses PHI_SEED0 + k
N_PHI = 2


def top(x, k):
    idx = np.sort(np.argsort(-np.abs(x))[:k])
    return idx.tolist(), x[idx].tolist()


def main():
    batch = synthetic.make_batch()
    members = []
    t0 = time.time()
    for k, s in enumerate(batch):
        t1 = time.time()
        b = Basis(s.grid, s.cell)
        m = {"k": k, "name": s.name, "grid": list(s.grid), "n_pw": b.n_pw, "n_occ": s.n_occ,
             "n_pdep": s.n_pdep}
        if s.grid[0] <= 32:
            ks = ks_states(b, s.v_r, s.n_occ)
            m["eps"] = ks.eps[: s.n_occ + 1].tolist()
            lam = pdep_reference(chi0bar_dense(b, ks), s.n_pdep)[0]
            m["pdep_eigenvalues"] = np.asarray(lam).tolist()
        else:
            ks = it.ks_states_lanczos(b, s.v_r, s.n_occ, tol=1e-14)
            m["eps"] = ks.eps[: s.n_occ + 1].tolist()
            phi = synthetic.random_vectors(PHI_SEED0 + k, N_PHI, b.n_pdep_dim)
            phi /= np.linalg.norm(phi, axis=1)[:, None]
            chi = it.chi0bar_apply_pcg(b, ks, s.v_r, phi, tol=1e-12)
            m["chi0"] = {"seed": PHI_SEED0 + k, "n": N_PHI, "M": (phi @ chi.T).tolist(),
                         "norm": np.linalg.norm(chi, axis=1).tolist(),
                         "idx": [], "val": []}
            for j in range(N_PHI):
                i, v = top(chi[j], 32)
                m["chi0"]["idx"].append(i)
                m["chi0"]["val"].append(v)
        members.append(m)
        print(f"member {k} ({s.grid[0]}^3, n_occ {s.n_occ}): {time.time() - t1:.0f} s", flush=True)
    out = {"what": "oracle reference values for the 32-member uneven batch "
                   "(written by tests/golden/make_batch_golden.py from oracle/ alone)",
           "members": members}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
