"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, by patching a
function for the duration of the test) and checks that the pin meant to
guard that step now fails.
"""
import contextlib

import numpy as np
import pytest

import problems as P
from oracle import ssamg as O

import test_oracle as T


@contextlib.contextmanager
def patched(name, fn):
    old = getattr(O, name)
    setattr(O, name, fn)
    try:
        yield old
    finally:
        setattr(O, name, old)


def _fails(check, *args):
    with pytest.raises((AssertionError, FloatingPointError, np.linalg.LinAlgError)):
        check(*args)


def test_sign_of_interpolation():
    orig = O.interpolation
    with patched("interpolation", lambda lev, p, d: tuple(-w for w in orig(lev, p, d))):
        _fails(T.test_interp_closed_forms_isotropic)


def test_interpolation_numerator_plane():
    orig = O.interpolation

    def swapped(lev, p, d):
        PW, PE = orig(lev, p, d)
        return PE, PW          # weights attached to the wrong neighbours
    with patched("interpolation", swapped):
        _fails(T._hierarchy_checks, T.chain([5, 7], [[1, .3, .1], [.2, 1, .4]]))


def test_galerkin_dropped_term():
    orig = O.galerkin_structured

    def dropped(fine, coarse, p):
        out = orig(fine, coarse, p)
        out[(0, 0, 0)] = out[(0, 0, 0)] * (1 + 1e-9)
        return out
    with patched("galerkin_structured", dropped):
        _fails(T._hierarchy_checks, P.laplace7(6))


def test_galerkin_unstructured_dropped():
    orig = O.galerkin_unstructured

    def half(fine, coarse):
        r, c, v, b = orig(fine, coarse)
        return r, c, 0.5 * v, b
    with patched("galerkin_unstructured", half):
        _fails(T._hierarchy_checks, P.multipart_aniso(m=4, layout=(2, 1, 1), seed=7))


def test_relaxation_weight_formula():
    with patched("relaxation_weight", lambda W, d, n: 2.0 / (3.0 + 0.0 * W[0])):
        _fails(T.test_omega_closed_forms)


def test_coupling_sum_wrong_entries():
    def wrong(lev):
        c = np.zeros((lev.nparts, 3))
        for p in range(lev.nparts):
            for d in range(3):
                c[p, d] = -sum(float(np.sum(a)) for o, a in lev.S[p].items() if o[d] == 0 and o != (0, 0, 0))
        return c
    with patched("coupling_sums", wrong):
        _fails(T.test_coupling_sums_closed_form)


def test_vcycle_without_post_smoothing():
    def pre_only(h, b, l=0):
        if l == h.L:
            return O._coarse_solve(h, b)
        lev = h.levels[l]
        x = lev.Dinv * b
        r = b - O.matvec(lev, x)
        bc = O.restrict(lev, r, h.levels[l + 1].n)
        return x + O.prolong(lev, pre_only(h, bc, l + 1))
    with patched("vcycle", pre_only):
        _fails(T.test_vcycle_symmetric_positive, P.multipart_aniso(m=4, layout=(2, 1, 1), seed=7))


def test_direction_tie_break():
    def largest_index(Wp, extent, ndim):
        cand = [d for d in range(ndim) if extent[d] > 1] or list(range(ndim))
        best = cand[-1]
        for d in reversed(cand):
            if Wp[d] < Wp[best]:
                best = d
        return best
    with patched("choose_direction", largest_index):
        _fails(T.test_isotropic_direction_cycles)


def test_part_boundary_fix_missing():
    orig = O.interpolation

    def nofix(lev, p, d):
        saved = lev.u_bits
        lev.u_bits = np.zeros_like(saved)
        try:
            return orig(lev, p, d)
        finally:
            lev.u_bits = saved
    with patched("interpolation", nofix):
        _fails(T.test_part_boundary_fix_row_sum_one)


def test_gradient_sign():
    orig = O.diffusion_exp_gradient
    with patched("diffusion_exp_gradient", lambda g, lam, x: -orig(g, lam, x)):
        _fails(T.test_diffusion_gradient_matches_finite_difference)


def _l1_smoother(factor_default, with_u):
    """The L1 branch of smoother_inverse with a planted mistake."""
    def fn(lev, params):
        out = np.zeros(lev.n)
        l1u = np.zeros(lev.n)
        if with_u and len(lev.u_val):
            np.add.at(l1u, lev.u_row, np.abs(lev.u_val))
        for p in range(lev.nparts):
            dv = lev.part_view(out, p)
            w = params.relax_factor if params.relax_factor > 0 else factor_default
            s = lev.part_view(l1u, p).copy()
            for a in lev.S[p].values():
                s += np.abs(a)
            dv[...] = w / s
        return out
    return fn


def test_l1_default_factor_one():
    with patched("smoother_inverse", _l1_smoother(1.0, True)):
        _fails(T.test_l1_jacobi_closed_form_interior_row)


def test_l1_row_sum_without_couplings():
    with patched("smoother_inverse", _l1_smoother(1.5, False)):
        _fails(T.test_l1_jacobi_row_sum_includes_couplings)


def test_skip_literal_in_place_of_rounds():
    orig = O.skipped_parts
    with patched("skipped_parts", lambda ds, nd, l, mode=1: orig(ds, nd, l, 2)):
        _fails(T.test_skip_isotropic_relaxes_on_full_coarsening_grids)
    with patched("skipped_parts", lambda ds, nd, l, mode=1: orig(ds, nd, l, 2)):
        _fails(T.test_skip_anisotropic_part_relaxes_while_direction_repeats)


def test_skip_relaxes_on_last_level_of_round():
    """Relaxation kept on the last level of each round instead of the first."""
    orig = O.skipped_parts

    def last_of_round(ds, nd, l, mode=1):
        if mode != 1:
            return orig(ds, nd, l, mode)
        nxt = orig(ds, nd, l + 1, 1) if l + 1 < len(ds) else [False] * len(ds[l])
        return [not n for n in nxt]
    with patched("skipped_parts", last_of_round):
        _fails(T.test_skip_isotropic_relaxes_on_full_coarsening_grids)
