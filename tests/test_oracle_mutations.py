"""Planted mistakes in the oracle must fail its pins.

Each test plants one plausible slip, replacing an oracle function with a wrong copy
for the duration of the test, and runs an existing pin against it. The slips are a
wrong sign, a dropped term, a wrong index or site, a transposed or missing adjoint,
and swapped projectors. If the pin still passed, it would not be guarding that part
of the oracle. The planted mistakes live only here, on the CPU; nothing on the CUDA
path is touched.
"""
import numpy as np
import pytest

import oracle
import oracle.cgne
import oracle.dwf
import oracle.force
import oracle.schur
import oracle.wilson
from oracle.lattice import ID4, P_MINUS, P_PLUS, colour_mul, dagger, norm2, spin_mul

import test_oracle_dwf as pins_dwf
import test_oracle_force as pins_force
import test_oracle_schur as pins_schur
import test_oracle_wilson as pins_wilson


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# --- Eq. wilson -------------------------------------------------------------------

def test_projector_sign_flip_is_caught(monkeypatch):
    """(1 + gamma_mu) on the forward hop and (1 - gamma_mu) on the backward one."""
    monkeypatch.setattr(oracle.wilson, "GAMMA", [-g for g in oracle.wilson.GAMMA])
    _fails(pins_wilson.test_free_field_closed_form, 1.0)


def test_missing_link_adjoint_is_caught(monkeypatch):
    """U_mu(x - mu) instead of U_mu(x - mu)^dagger on the backward hop."""
    monkeypatch.setattr(oracle.wilson, "dagger", lambda u: u)
    _fails(pins_wilson.test_gamma5_hermiticity_and_adjoint, 1.0)


def test_backward_link_from_wrong_site_is_caught(monkeypatch):
    """U_mu(x)^dagger instead of U_mu(x - mu)^dagger on the backward hop."""
    shift = oracle.wilson._shift

    def hop(psi, U, dagger_op=False, bc_t=1.0):
        lead = psi.ndim - 6
        sg = -1.0 if dagger_op else 1.0
        out = np.zeros_like(psi)
        for mu in range(4):
            umu = U[..., mu, :, :]
            out += spin_mul(ID4 - sg * oracle.wilson.GAMMA[mu],
                            colour_mul(umu, shift(psi, lead, mu, +1, bc_t)))
            out += spin_mul(ID4 + sg * oracle.wilson.GAMMA[mu],
                            colour_mul(dagger(umu), shift(psi, lead, mu, -1, bc_t)))
        return out

    monkeypatch.setattr(oracle.wilson, "hop", hop)
    _fails(pins_wilson.test_gamma5_hermiticity_and_adjoint, 1.0)


# --- Eq. mobius1, Eq. eqP ------------------------------------------------------------

def test_dropped_mass_corners_are_caught(monkeypatch):
    """The corner blocks -m D_{1-} P_+ and -m D_{Ls-} P_- left out."""
    blocks = oracle.dwf.blocks

    def no_corners(Ls, alpha, m):
        return [b for b in blocks(Ls, alpha, m) if not (abs(b[0] - b[1]) == Ls - 1 and Ls > 2)]

    monkeypatch.setattr(oracle.dwf, "blocks", no_corners)
    _fails(pins_dwf.test_alpha1_is_standard_mobius, "mobius")


def test_alpha_on_wrong_projector_is_caught(monkeypatch):
    """Row 1 diagonal D_{1+}(P_+ + alpha P_-) instead of D_{1+}(P_- + alpha P_+):
    invisible at alpha = 1, caught by D_alpha P = D_1 P A at alpha != 1."""
    blocks = oracle.dwf.blocks

    def swapped(Ls, alpha, m):
        out = list(blocks(Ls, alpha, m))
        out[0] = (0, 0, "+", P_PLUS + alpha * P_MINUS)
        return out

    monkeypatch.setattr(oracle.dwf, "blocks", swapped)
    pins_dwf.test_alpha1_is_standard_mobius("mobius")  # alpha = 1 cannot see it
    _fails(pins_dwf.test_dalpha_p_equals_d1_p_a, "mobius", 0.5)


def test_swapped_projectors_in_p_are_caught(monkeypatch):
    """(P v)_s = P_+ v_s + P_- v_{s+1} instead of Eq. eqP."""
    def p_apply(v):
        return spin_mul(P_PLUS, v) + spin_mul(P_MINUS, np.roll(v, -1, axis=0))

    monkeypatch.setattr(oracle, "p_apply", p_apply)
    _fails(pins_dwf.test_dalpha_p_equals_d1_p_a, "mobius", 1.25)


def test_shifted_p_inverse_is_caught(monkeypatch):
    """P^-1 rolling the wrong way (the index slip s+1 for s-1)."""
    def p_inverse(w):
        return spin_mul(P_MINUS, w) + spin_mul(P_PLUS, np.roll(w, -1, axis=0))

    monkeypatch.setattr(oracle, "p_inverse", p_inverse)
    _fails(pins_dwf.test_p_inverse_and_ls2_blocks)


# --- Eq. redblack -------------------------------------------------------------------

def test_i_for_i_inverse_in_schur_is_caught(monkeypatch):
    """D_bb = 1 - I D_br I^-1 D_rb (the outer I^-1 replaced by I), with its adjoint
    planted consistently: the adjoint identity still holds, the Schur-complement
    definition (the black rows of D_alpha give I D_bb) does not."""
    S = oracle.schur.DWFSystem

    def dbb(self, hb):
        return hb - self.apply_local_matrix(self.local_matrix(),
                                            self.d_br(self.iinv(self.d_rb(hb))))

    def dbb_dag(self, hb):
        return hb - self.d_rb_dag(self.iinv_dag(self.d_br_dag(
            self.apply_local_matrix(np.conj(self.local_matrix().T), hb))))

    monkeypatch.setattr(S, "dbb", dbb)
    monkeypatch.setattr(S, "dbb_dag", dbb_dag)
    _fails(pins_schur.test_dbb_adjoint_and_definition)


def test_adjoint_factor_order_is_caught(monkeypatch):
    """D_bb^+ with its factors in the forward order instead of reversed."""
    S = oracle.schur.DWFSystem

    def dbb_dag(self, hb):
        return hb - self.iinv_dag(self.d_br_dag(self.iinv_dag(self.d_rb_dag(hb))))

    monkeypatch.setattr(S, "dbb_dag", dbb_dag)
    _fails(pins_schur.test_dbb_adjoint_and_definition)


# --- CGNR ---------------------------------------------------------------------------

def test_cgnr_wrong_sign_update_is_caught(monkeypatch):
    """x -= a p instead of x += a p (a sign slip in the solution update)."""
    def cgnr(apply_d, apply_ddag, rhs, tol=1e-10, maxiter=2000, check_every=10):
        bnorm = np.sqrt(norm2(rhs))
        x = np.zeros_like(rhs)
        r = rhs.copy()
        z = apply_ddag(r)
        p = z.copy()
        zz = norm2(z)
        res = 1.0
        for it in range(1, 2001):
            w = apply_d(p)
            a = zz / norm2(w)
            x = x - a * p
            r = r - a * w
            if it % check_every == 0:
                r = rhs - apply_d(x)
                res = np.sqrt(norm2(r)) / bnorm
                if res <= tol:
                    break
            z = apply_ddag(r)
            zz_new = norm2(z)
            p = z + (zz_new / zz) * p
            zz = zz_new
        return x, it, res

    monkeypatch.setattr(oracle, "cgnr", cgnr)
    _fails(pins_schur.test_cgnr_random_dense)


# --- force --------------------------------------------------------------------------

def test_transposed_force_outer_product_is_caught(monkeypatch):
    """The link outer product eta xi^+ transposed in colour."""
    outer = oracle.force._outer
    monkeypatch.setattr(oracle.force, "_outer", lambda a, b: np.swapaxes(outer(a, b), -1, -2))
    _fails(pins_force.test_force_vs_finite_differences_raw_entries)


# --- App. A overlap, row scaling, single-site evaluator ------------------------------

def test_sign_function_flip_is_caught(monkeypatch):
    """eps of Eq. polar with the two products exchanged (eps -> -eps)."""
    import oracle.overlap
    tanh_form = oracle.overlap.sign_tanh_form
    monkeypatch.setattr(oracle.overlap, "sign_tanh_form",
                        lambda dwm, g5, b, c: -tanh_form(dwm, g5, b, c))
    _fails(pins_schur.test_propagator_equals_overlap_inverse, "mobius", 1.0)


def test_row_scaling_condition_reversed_is_caught(monkeypatch):
    """Rows scaled where b_s + c_s < 1 instead of > 1."""
    def row_scale(self):
        a = self.b + self.c
        return np.where(a < 1.0, 1.0 / a, 1.0)

    monkeypatch.setattr(oracle.schur.DWFSystem, "row_scale", row_scale)
    _fails(pins_schur.test_row_scale_factors)


def test_pointwise_neighbour_direction_is_caught(monkeypatch):
    """The single-site evaluator stepping to x - mu where it means x + mu."""
    import oracle.pointwise
    import test_oracle_pointwise as pins_pointwise
    shift = oracle.pointwise._SiteOps._shift
    monkeypatch.setattr(oracle.pointwise._SiteOps, "_shift",
                        lambda self, c, mu, d: shift(self, c, mu, -d))
    _fails(pins_pointwise.test_pointwise_matches_whole_lattice, 1.0, 0)
