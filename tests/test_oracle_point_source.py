"""Pins of the oracle's point-source scattering (the rigid-sphere comparison
of Sec. 5.2, source at (-2, 0, 0)): the closed form against the Mie series
as the source recedes, and the oracle's dense solution converging to the
closed form for both signs of the coupling."""
import numpy as np
import pytest

import oracle
from inputs import icosphere


def test_closed_form_tends_to_plane_wave_mie():
    """|x_s| -> infinity: G(x, x_s) -> e^{ik r_s}/(4 pi r_s) e^{ik d.x} with
    d = -x_s/r_s, so the surface field tends to the Mie series times that
    amplitude (relative gap O(n^2/(k r_s)))."""
    k = 3.0
    ct = np.linspace(-1.0, 1.0, 9)  # cos of the angle to d; the angle to x_s is its negative
    gaps = []
    for rs in (1e5, 1e7):
        u = oracle.point_source_surface_field(k, rs, -ct, nmax=60)
        m = oracle.mie_surface_field(k, ct) * np.exp(1j * k * rs) / (4 * np.pi * rs)
        gaps.append(np.abs(u - m).max() / np.abs(m).max())
    assert gaps[1] < 1e-6 and gaps[1] < gaps[0] / 50


def test_closed_form_series_converged():
    ct = np.linspace(-1.0, 1.0, 11)
    for k in (5.0, 20.0):
        a = oracle.point_source_surface_field(k, 2.0, ct)
        b = oracle.point_source_surface_field(k, 2.0, ct, nmax=200)
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("alpha_sign", [1.0, -1.0])
def test_dense_solution_converges_to_closed_form(alpha_sign):
    k, src = 5.0, np.array([-2.0, 0.0, 0.0])
    errs = []
    for L in (2, 3, 4):
        v, f = icosphere(L)
        c, *_ = oracle.geometry(v, f)
        a = oracle.assemble(v, f, k, alpha_sign=alpha_sign)
        b = oracle.rhs_point_source(v, f, k, [src], alpha_sign=alpha_sign)[0]
        u = oracle.lu_solve(a, b)
        cg = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ (src / np.linalg.norm(src))
        ue = oracle.point_source_surface_field(k, 2.0, cg)
        errs.append(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    assert errs[2] < errs[1] / 2 < errs[0] / 4
    assert errs[2] < 1e-2
