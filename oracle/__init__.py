"""Plain FP64 CPU oracle of the alpha-Mobius domain-wall method (arXiv:1501.04950).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline legs of bench.py may import this package; the library under
paper_1501_04950_gb300/ never does.  The oracle shares no code with the CUDA
path: it takes the same seeded inputs (module synthetic) and states the
paper's formulas literally in numpy, complex128 throughout.

Modules and the passages they follow:
  lattice  gamma matrices (chiral basis), checkerboard, half-field layout
  wilson   D_w(M5), Sec. 2 Eq. wilson (and its adjoint)
  dwf      D_alpha(m), Sec. 2 Eq. mobius1 / Eq. coeff; P (App. A Eq. eqP); A
  schur    I, D_rb, D_br, D_bb and D_bb^+, Sec. 3 Eq. redblack
  cgne     CG on the normal equations, Sec. 3; propagator Eq. tosolve1, App. B;
           D_OV(m) b through the mass-exchanged 5D solve
  force    dS/dU for S = phi^+ (D_bb^+ D_bb)^-1 phi (adjoint of Eq. redblack)
  overlap  dense D_OV with the tanh form of eps, App. A Eq. polar / argument

Every function is pinned by tests/test_oracle_*.py against closed forms,
identities stated in the paper, brute-force dense solves and finite
differences.
"""
from .lattice import (GAMMA, GAMMA5, P_MINUS, P_PLUS, full_to_half, half_to_full,
                      norm2, parity_grid, shape4, vdot, volume)
from .wilson import dw, hop
from .dwf import (a_apply, blocks, dalpha, dalpha_dag, dalpha_generic, mobius_standard,
                  p_apply, p_inverse)
from .schur import DWFSystem
from .cgne import (cgnr, overlap_apply, propagator_rhs, solve_propagator, source_5d,
                   propagator_from_psi)
from .force import action, cg_normal, force_gradient, su3_force, traceless_antihermitian
from . import overlap

__all__ = [
    "GAMMA", "GAMMA5", "P_MINUS", "P_PLUS", "full_to_half", "half_to_full", "norm2",
    "parity_grid", "shape4", "vdot", "volume", "dw", "hop", "a_apply", "blocks",
    "dalpha", "dalpha_dag", "dalpha_generic", "mobius_standard", "p_apply", "p_inverse",
    "DWFSystem", "cgnr", "overlap_apply", "propagator_rhs", "solve_propagator", "source_5d",
    "propagator_from_psi", "action", "cg_normal", "force_gradient", "su3_force",
    "traceless_antihermitian", "overlap",
]
