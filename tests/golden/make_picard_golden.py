"""Write golden records of oracle solves, from the CPU oracle only.

  python tests/golden/make_picard_golden.py small
      the oracle's truncated inexact Picard iteration (Algorithm 3.1) on a preset:
      tests/golden/picard_<preset>.txt (iteration counts, ||u||, ||p||, the final
      relative residual, the full-tensor values of u and p at 256 seeded index
      triples) and tests/golden/picard_<preset>_cores.npz (the cores of u and p,
      for comparisons by TT difference);
  python tests/golden/make_picard_golden.py medium --stokes
      the Stokes initial solve of Algorithm 3.1 (TT-GMRES with the mean-based LSC
      preconditioner, Section 5.2) on a preset: tests/golden/stokes_<preset>.npz
      (cores, outer and inner iteration counts, ||f||, the truncated residual).
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


def stokes(name):
    import time
    from oracle.solver import MeanLSC, gmres, _Pair
    prob = synth.preset(name)
    d = Discretisation(prob)
    t = prob.tol
    fu, fp = d.rhs()
    fnorm = float(np.hypot(norm(fu), norm(fp)))
    P = MeanLSC(d, None, t.eps_gmres, t.tol_inner, t.maxit_inner)
    t0 = time.time()
    (u, p), st = gmres(lambda v: d.apply(None, *v), P, (fu, fp), tol=t.tol_gmres, eps=t.eps_gmres,
                       maxit=t.maxit_gmres, space=_Pair, bnorm=fnorm)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"stokes_{name}.npz")
    np.savez_compressed(out, u1=u.z1, u2=u.z2, u3=u.z3, p1=p.z1, p2=p.z2, p3=p.z3, its=st["its"],
                        inner_its=np.array(P.inner_its), fnorm=fnorm, res=st["res"][-1],
                        seconds=time.time() - t0)
    print(out, st["its"], P.inner_its, u.ranks, p.ranks)


def main(name):
    prob = synth.preset(name)
    d = Discretisation(prob)
    u, p, st = picard(d)
    np.savez_compressed(os.path.join(os.path.dirname(os.path.abspath(__file__)), f"picard_{name}_cores.npz"),
                        u1=u.z1, u2=u.z2, u3=u.z3, p1=p.z1, p2=p.z2, p3=p.z3)
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
    name = sys.argv[1] if len(sys.argv) > 1 else "small"
    if "--stokes" in sys.argv:
        stokes(name)
    else:
        main(name)
