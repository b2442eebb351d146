"""The exact fields of the paper's Examples 5.2 and 5.3 (Sec. 5.1): divergence
free, and the forcing equals -Lap u + grad p, both checked against sympy's
symbolic derivatives of the printed fields (skipped where sympy is absent)."""
import numpy as np
import pytest

import kfbim_inputs as ki

sp = pytest.importorskip("sympy")
x, y, z = sp.symbols("x y z")
FIELDS = {
    "5.2": ([2 * x**3 * y / 3 - z**2 * x**2 + sp.exp(z) + sp.sin(sp.pi * z),
             -x**2 * y**2 + sp.cos(sp.pi * x),
             2 * z**3 * x / 3 + sp.exp(x) + sp.sin(sp.pi * x)],
            (x - 1) ** 3 * (y - 1) ** 3 * (z - 1) ** 3,
            ki.example52_velocity, ki.example52_pressure, ki.example52_forcing),
    "5.3": ([-4 * x * y * (1 - x**2 - y**2) - x**2 * (x**2 + 6 * z**2 - 2) + z**2 * (3 * z**2 - 2)
             + sp.exp(sp.cos(y)) + sp.exp(sp.sin(z)),
             x**2 * (3 * x**2 - 6 * y**2 - 2) - y**2 * (y**2 - 2) + sp.exp(sp.sin(x)),
             -4 * (1 - x**2 - z**2) * x * z + sp.exp(sp.cos(x))],
            sp.exp(1 - y**2 - z**3) * sp.sin(x**2 + 1),
            ki.example53_velocity, ki.example53_pressure, ki.example53_forcing),
}


@pytest.mark.parametrize("key", sorted(FIELDS))
def test_fields_against_symbolic_derivatives(key):
    U, p, fu, fp, ff = FIELDS[key]
    assert sp.simplify(sum(sp.diff(U[i], v) for i, v in enumerate((x, y, z)))) == 0
    P = np.random.default_rng(1).uniform(-1.1, 1.1, (50, 3))
    args = (P[:, 0], P[:, 1], P[:, 2])
    u = np.stack([sp.lambdify((x, y, z), U[i])(*args) for i in range(3)], -1)
    f = np.stack([sp.lambdify((x, y, z), -sum(sp.diff(U[i], v, 2) for v in (x, y, z))
                              + sp.diff(p, (x, y, z)[i]))(*args) for i in range(3)], -1)
    assert np.abs(fu(P) - u).max() <= 1e-13 * np.abs(u).max()
    assert np.abs(fp(P) - sp.lambdify((x, y, z), p)(*args)).max() <= 1e-13 * np.abs(fp(P)).max()
    assert np.abs(ff(P) - f).max() <= 1e-13 * np.abs(f).max()


NAVIER = {
    "5.4": [sp.sin(2 * sp.pi * (x**2 + y**2 + z**2)) * sp.cos(2 * y) * sp.cos(z),
            sp.sin(2 * sp.pi * (x**2 + y**2 + z**2)) * sp.cos(x) * sp.cos(x + z),
            sp.sin(2 * sp.pi * (x**2 + y**2 + z**2)) * sp.cos(sp.pi * x) * sp.cos(y)],
    "5.5": [x**2 + y**2 + z**2 - 4 + sp.cos(x) * sp.cos(y) * sp.cos(z),
            x**2 + y**2 + z**2 - 4 + x * y + sp.cos(x) * sp.cos(y) * sp.cos(z),
            x**2 + y**2 + z**2 - 4 + y * z + sp.cos(x) * sp.cos(y) * sp.cos(z)],
    "5.6": [sp.exp(1 - y**2 - z**2) * sp.sin(3 * x**2 + 2), sp.sin(1 - x**2 - y**2 - z**2),
            3 * x**2 + 2 * y**2 + z**2],
}


@pytest.mark.parametrize("key", sorted(NAVIER))
def test_navier_fields_against_symbolic_derivatives(key):
    U = NAVIER[key]
    _, E, nu = ki.NAVIER_EXAMPLES[key]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    div = sum(sp.diff(U[i], v) for i, v in enumerate((x, y, z)))
    P = np.random.default_rng(2).uniform(-1.1, 1.1, (40, 3))
    args = (P[:, 0], P[:, 1], P[:, 2])
    u = np.stack([sp.lambdify((x, y, z), U[i])(*args) for i in range(3)], -1)
    f = np.stack([sp.lambdify((x, y, z), -mu * sum(sp.diff(U[i], v, 2) for v in (x, y, z))
                              - (lam + mu) * sp.diff(div, (x, y, z)[i]))(*args) for i in range(3)], -1)
    assert np.abs(ki.navier_example_displacement(key, P) - u).max() <= 1e-13 * np.abs(u).max()
    assert np.abs(ki.navier_example_forcing(key, P) - f).max() <= 1e-12 * np.abs(f).max()
