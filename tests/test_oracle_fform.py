"""The h-form oracle against the literal f-form of the paper's equations (oracle/fform.py).

The f-form stores f, takes the equilibrium of Eq. (5) with the division by rho of Eqs. (6)-(7)
and the wall populations of Eqs. (8)-(9) as printed; the h-form oracle (lbm_oracle.c) marches
the perturbation h = (f - w) / u_ref with the equivalent linear forms.  The two agree up to
the f-form's cancellation (here within 1e-11 of the field), and planted mistakes in the h-form's wall,
transport and relaxation code each break the agreement."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import march as q
from oracle.fform import make_fform_problem
from oracle.march import CAVITY, COUETTE, make_problem

CASES = [
    # kind, n, geom, nx, ny, kn, u_bottom, u_top
    ("half", 4, COUETTE, 1, 24, 0.1, 0.01, -0.01),      # plates moving in opposite directions
    ("half", 2, COUETTE, 4, 9, 0.05, -0.01, 0.01),      # periodic columns
    ("half", 4, CAVITY, 9, 7, 0.1, 0.003, 0.01),        # moving bottom and lid, nx != ny
    ("full", 3, CAVITY, 8, 6, 0.2, 0.0, 0.01),          # D2Q9 (xi = 0 row and column)
    ("full", 4, CAVITY, 7, 7, 0.3, 0.0, 0.01),          # D2Q16
    ("half", 6, CAVITY, 5, 4, 0.05, 0.0, 0.02),         # D2Q^h_144
]
IDS = ["couette-h64", "couette-periodic-h16", "cavity-h64-9x7", "cavity-D9", "cavity-D16", "cavity-h144"]
TOL = 1e-11          # measured: 1e-15 to 2e-14 after 6 steps, 3e-13 after 600


def _pair(case, seed=11):
    kind, n, geom, nx, ny, kn, ub, ut = case
    p = make_problem(kind, n, geom, nx, ny, kn, ub, ut)
    f = make_fform_problem(kind, n, geom, nx, ny, kn, ub, ut)
    h0 = np.random.default_rng(seed).standard_normal((p.n, p.ncells))
    return p, f, h0


def _fform_steps(fp, p, h0, steps):
    u_ref = p.coeffs["u_ref"]
    f = (p.w[:, None] + u_ref * h0).reshape(p.n, p.ny, p.nx)
    for _ in range(steps):
        f = fp.step(f)
    return (f.reshape(p.n, p.ncells) - p.w[:, None]) / u_ref


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_h_form_matches_literal_f_form(case):
    p, fp, h0 = _pair(case)
    assert fp.dt == pytest.approx(p.coeffs["dt"], rel=1e-15) and fp.omega == pytest.approx(p.coeffs["omega"], rel=1e-15)
    steps = 6
    got = p.step(h0, steps)
    ref = _fform_steps(fp, p, h0, steps)
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


def test_h_form_matches_literal_f_form_over_a_long_march():
    """A cold-start cavity marched 600 steps: the two forms stay within the f-form's
    cancellation error."""
    case = ("half", 4, CAVITY, 12, 12, 0.1, 0.0, 0.01)
    p, fp, _ = _pair(case)
    zero = np.zeros((p.n, p.ncells))
    got = p.step(zero, 600)
    ref = _fform_steps(fp, p, zero, 600)
    assert np.abs(got).max() > 0.01                 # the flow has developed
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


# --- planted mistakes in the h-form oracle: each must break the agreement with the f-form

MUTANTS = {
    "wall driving term dropped": ("return p->w[a] * (rho_w * (1.0 + xt * u) + xt * u / c->u_ref);",
                                  "return p->w[a] * (rho_w * (1.0 + xt * u));"),
    "wall speed sign in the ghost": ("return p->w[a] * (rho_w * (1.0 + xt * u) + xt * u / c->u_ref);",
                                     "return p->w[a] * (rho_w * (1.0 - xt * u) + xt * u / c->u_ref);"),
    "wall density normaliser doubled": ("return s / d;", "return s / (2.0 * d);"),
    "outgoing populations in the wall density": ("if (xn < 0) s += -xn * h[(long)a * ncells + cell];",
                                                 "if (xn > 0) s += xn * h[(long)a * ncells + cell];"),
    "x Courant number with dy": ("double nux = fabs(p->xi_x[a]) * c->dt / c->dx;",
                                 "double nux = fabs(p->xi_x[a]) * c->dt / c->dy;"),
    "x upwind cell on the wrong side": ("if (x > 0) hx = ha[cell - 1];", "if (x > 0) hx = ha[cell + (x < nx - 1 ? 1 : 0)];"),
    "j_y dropped from the equilibrium": ("(rho + p->xi_x[a] * jx + p->xi_y[a] * jy);\n        out[a] = hs[a]",
                                         "(rho + p->xi_x[a] * jx);\n        out[a] = hs[a]"),
    "relaxation rate halved": ("out[a] = hs[a] - c->omega * (hs[a] - heq);",
                               "out[a] = hs[a] - 0.5 * c->omega * (hs[a] - heq);"),
}


def _mutant_step(tmp_path, name, old, new):
    src_path = os.path.join(os.path.dirname(q.__file__), "lbm_oracle.c")
    with open(src_path) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"planted mistake {name!r}: the oracle text it replaces is not unique"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    c_file, so_file = tmp_path / f"{tag}.c", tmp_path / f"{tag}.so"
    c_file.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           str(c_file), "-o", str(so_file), "-lm"])
    lib = ctypes.CDLL(str(so_file))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, dp, dp]
    lib.orc_step.restype = None

    def step(p, h, steps):
        cur = np.ascontiguousarray(h, dtype=np.float64).copy()
        nxt = np.empty_like(cur)
        for _ in range(steps):
            lib.orc_step(ctypes.addressof(p._p), ctypes.addressof(p._c), cur.ctypes.data_as(dp), nxt.ctypes.data_as(dp))
            cur, nxt = nxt, cur
        return cur
    return step


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_breaks_the_f_form_agreement(tmp_path, name):
    step = _mutant_step(tmp_path, name, *MUTANTS[name])
    caught = []
    for case, cid in zip(CASES, IDS):
        p, fp, h0 = _pair(case)
        got = step(p, h0, 6)
        ref = _fform_steps(fp, p, h0, 6)
        if not np.abs(got - ref).max() <= TOL * np.abs(ref).max():
            caught.append(cid)
    assert caught, f"planted mistake {name!r} agrees with the literal f-form on every case"
