"""The pins hold the oracle to the paper: each plausible mistake planted in a
copy of the oracle's C source (a dropped term, a wrong sign, factor or index, a
transposed operand) makes at least one pin of tests/test_oracle_*.py fail.

Each mutant is compiled on its own and the pin files run against it in a child
process (the oracle module loads the mutant through VANS_ORACLE_MUTANT_LIB);
the real oracle is never modified.  CPU only."""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vans_oracle.c")
PINS = ["tests/test_oracle_cell.py", "tests/test_oracle_flows.py", "tests/test_oracle_adjoint.py",
        "tests/test_oracle_flux.py"]

# name, text in the oracle, planted mistake (each text occurs exactly once)
MUTANTS = [
    ("lattice: a D2Q9 weight", "    4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,",
     "    4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 8,"),
    ("lattice: a D3Q19 velocity component", "{0, 1, -1}, {0, -1, 1}};", "{0, 1, -1}, {0, -1, -1}};"),
    ("moments: no half on the body force (Eq. 1moment)",
     "c->m[k] = c->j[k] + 0.5 * c->Pc[k] + 0.5 * c->R * gcomp(p, L, k);",
     "c->m[k] = c->j[k] + 0.5 * c->Pc[k] + c->R * gcomp(p, L, k);"),
    ("moments: pressure gradient dropped from Eq. 1moment",
     "c->m[k] = c->j[k] + 0.5 * c->Pc[k] + 0.5 * c->R * gcomp(p, L, k);",
     "c->m[k] = c->j[k] + 0.5 * c->R * gcomp(p, L, k);"),
    ("moments: p = rho instead of cs^2 rho", "c->Pc[k] = CS2 * c->rho * gradc[k];",
     "c->Pc[k] = c->rho * gradc[k];"),
    ("drag: Darcy term with the wrong sign",
     "c->F[k] = c->R * gcomp(p, L, k) - c->alpha * c->u[k] - c->beta * c->un * c->u[k];",
     "c->F[k] = c->R * gcomp(p, L, k) + c->alpha * c->u[k] - c->beta * c->un * c->u[k];"),
    ("drag: Forchheimer term dropped",
     "c->F[k] = c->R * gcomp(p, L, k) - c->alpha * c->u[k] - c->beta * c->un * c->u[k];",
     "c->F[k] = c->R * gcomp(p, L, k) - c->alpha * c->u[k];"),
    ("drag: Ergun K with (1 - eps) once", "a = c * (1 - eps) * (1 - eps) / eps;",
     "a = c * (1 - eps) / eps;"),
    ("drag: F_eps power of eps", "const double Feps = 1.75 / sqrt(150.0 * eps * eps * eps);",
     "const double Feps = 1.75 / sqrt(150.0 * eps * eps);"),
    ("velocity: wrong factor in the quadratic solve",
     "const double D = a + sqrt(a * a + 4.0 * b * mm);",
     "const double D = a + sqrt(a * a + 2.0 * b * mm);"),
    ("equilibrium: quadratic term without its 1/2",
     "(1.0 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2));\n    }\n}",
     "(1.0 + eu / CS2 + eu * eu / (CS2 * CS2) - uu / (2 * CS2));\n    }\n}"),
    ("equilibrium: no eps weighting", "feq[i] = L->w[i] * eps * rho *", "feq[i] = L->w[i] * rho *"),
    ("sources: prefactor 1 - 1/(2 tau) dropped", "const double c = 1.0 - 1.0 / (2.0 * tau);",
     "const double c = 1.0;"),
    ("sources: e_i + u instead of e_i - u",
     "s += ((L->e[i][k] - u[k]) / CS2 + eu * L->e[i][k] / (CS2 * CS2)) * V[k];",
     "s += ((L->e[i][k] + u[k]) / CS2 + eu * L->e[i][k] / (CS2 * CS2)) * V[k];"),
    ("sources: P_i dropped (only F_i)", "c->V[k] = c->Pc[k] + c->F[k];", "c->V[k] = c->F[k];"),
    ("grad eps: stencil sign", "for (int k = 0; k < 3; ++k) G[k] += L->w[i] * L->e[i][k] * en;",
     "for (int k = 0; k < 3; ++k) G[k] -= L->w[i] * L->e[i][k] * en;"),
    ("grad eps: zero instead of eps(x) past a wall", "if (xs < 0 || ys < 0 || zs < 0) en = eps[n];",
     "if (xs < 0 || ys < 0 || zs < 0) en = 0.0;"),
    ("collision: tau multiplies instead of dividing",
     "f[i * N + n] = fc[i] - (fc[i] - feq[i]) / tau + S[i];",
     "f[i * N + n] = fc[i] - (fc[i] - feq[i]) * tau + S[i];"),
    ("streaming: bounce-back keeps the direction", "fn[L->opp[i] * N + n] = fs[i * N + n] - add;",
     "fn[i * N + n] = fs[i * N + n] - add;"),
    ("streaming: moving wall gain with the wrong sign", "add = 2.0 * L->w[i] * eps[n] * eu / CS2;",
     "add = -2.0 * L->w[i] * eps[n] * eu / CS2;"),
    ("plates on nodes: neighbour's non-equilibrium part dropped",
     "for (int i = 0; i < L->q; ++i) f[i * N + nb_] = feqb[i] + (fc[i] - feqf[i]);",
     "for (int i = 0; i < L->q; ++i) f[i * N + nb_] = feqb[i];"),
    ("adjoint: Darcy partial of u with the wrong sign",
     "ubar[k] += -c->alpha * Fbar[k] - c->beta * c->un * Fbar[k];",
     "ubar[k] += c->alpha * Fbar[k] - c->beta * c->un * Fbar[k];"),
    ("adjoint: eps partial of rho = R / eps dropped",
     "*epsbar += -rhobar * c->R / (eps * eps);", "*epsbar += 0.0 * rhobar;"),
    ("adjoint: transposed grad-eps stencil with the wrong sign", "epsbar[t] += s / CS2;",
     "epsbar[t] -= s / CS2;"),
    ("drag: fixed-K Forchheimer power of eps", "b = eps * eps * eps * p->F_eps / sqrt(p->K);",
     "b = eps * eps * p->F_eps / sqrt(p->K);"),
    ("velocity: |m| for every component", "for (int k = 0; k < 3; ++k) u[k] = 2.0 * m[k] / D;",
     "for (int k = 0; k < 3; ++k) u[k] = 2.0 * mm / D;"),
    ("streaming: periodic wrap off by one", "t = (t + n) % n;", "t = (t + n - 1) % n;"),
    ("plates on nodes: plate equilibrium with the fluid node's eps",
     "equilibrium(L, eps[nb_], c.rho, ub, feqb);", "equilibrium(L, eps[nf], c.rho, ub, feqb);"),
    ("plates on nodes: upper plate at rest",
     "equilibrium(L, eps[n], R / eps[n], y == 0 ? zero : p->u_wall, feq);",
     "equilibrium(L, eps[n], R / eps[n], zero, feq);"),
    ("flux: the populations' momentum without the half-force terms of Eq. 1moment",
     "s += c.R * c.u[0];", "s += c.j[0];"),
    ("flux: rho u_x instead of eps rho u_x", "s += c.R * c.u[0];", "s += c.rho * c.u[0];"),
    ("flux: the plane next to the outlet",
     "p->nx + x_out;\n            double fc[19], gc[3] = {grad[n], grad[N + n], grad[2 * N + n]};\n"
     "            cell_t c;",
     "p->nx + (x_out + 1) % p->nx;\n            double fc[19], gc[3] = {grad[n], grad[N + n], "
     "grad[2 * N + n]};\n            cell_t c;"),
    ("flux: the y component", "s += c.R * c.u[0];", "s += c.R * c.u[1];"),
]
# Not among them: the rule for a D3Q19 population that crosses the moving y
# wall and a z wall at once (reading R7 of the oracle: plain bounce-back).  The
# other choice converges to the same continuum flow, so no closed form can
# decide it; the GPU follows the oracle's choice and the parity tests hold it.


def _compile(src: str, out: str) -> None:
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    "-o", out, src, "-lm"], check=True, capture_output=True)


def _pins_fail(lib: str) -> bool:
    env = dict(os.environ, VANS_ORACLE_MUTANT_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", *PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    return r.returncode != 0


def test_every_mutant_is_caught():
    src = open(SRC).read()
    with tempfile.TemporaryDirectory() as tmp:
        libs = []
        for k, (name, old, new) in enumerate(MUTANTS):
            assert src.count(old) == 1, (name, src.count(old))
            path = os.path.join(tmp, f"m{k}.c")
            with open(path, "w") as fh:
                fh.write(src.replace(old, new))
            lib = os.path.join(tmp, f"m{k}.so")
            _compile(path, lib)
            libs.append(lib)
        with ThreadPoolExecutor(max_workers=4) as pool:
            caught = list(pool.map(_pins_fail, libs))
    survivors = [MUTANTS[k][0] for k, c in enumerate(caught) if not c]
    assert not survivors, survivors


def test_the_unmutated_source_passes_through_the_same_route():
    """The route itself (a copy compiled the same way, loaded through the
    variable) passes every pin, so a caught mutant is caught for its mistake."""
    with tempfile.TemporaryDirectory() as tmp:
        lib = os.path.join(tmp, "same.so")
        _compile(SRC, lib)
        assert not _pins_fail(lib)
