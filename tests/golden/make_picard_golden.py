"""Write tests/golden/picard_<preset>.txt from the CPU oracle only.

Runs the oracle's truncated inexact Picard iteration (Algorithm 3.1) on a
preset and stores: the iteration counts, ||u||, ||p||, the final relative
residual, and the full-tensor values of u and p at 256 seeded index triples
each.  GPU tests compare against these samples.

    python tests/golden/make_picard_golden.py small
"""
import os
import sys

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle.solver import picard  # noqa: E402
from oracle.system import Discretisation  # noqa: E402
from oracle.tt import norm  # noqa: E402


def entry(t, i, s, j):
    """z(i, s, j) = z1[i, :] z2[:, s, :] z3[:, j] (eq. z_tt)."""
    return float(t.z1[i] @ t.z2[:, s, :] @ t.z3[:, j])


def main(name):
    prob = synth.preset(name)
    d = Discretisation(prob)
    u, p, st = picard(d)
    rng = np.random.default_rng(2024)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"picard_{name}.txt")
    with open(out, "w") as f:
        f.write(f"# oracle Picard solution of the '{name}' preset (Algorithm 3.1, Table 5.2 tolerances)\n")
        f.write("# written by tests/golden/make_picard_golden.py from oracle/ only\n")
        f.write(f"picard_its {st['picard_its']}\n")
        f.write(f"stokes_its {st['stokes_its']}\n")
        f.write("gmres_its " + " ".join(str(k) for k in st["gmres_its"]) + "\n")
        f.write(f"rel_res {st['res'][-1] / st['fnorm']:.17e}\n")
        f.write(f"norm_u {norm(u):.17e}\n")
        f.write(f"norm_p {norm(p):.17e}\n")
        f.write(f"ranks_u {u.ranks[0]} {u.ranks[1]}\n")
        f.write(f"ranks_p {p.ranks[0]} {p.ranks[1]}\n")
        for tag, t in (("u", u), ("p", p)):
            n_t, n_xi, n_x = t.shape
            for _ in range(256):
                i, s, j = int(rng.integers(n_t)), int(rng.integers(n_xi)), int(rng.integers(n_x))
                f.write(f"{tag} {i} {s} {j} {entry(t, i, s, j):.17e}\n")
    print(out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "small")
