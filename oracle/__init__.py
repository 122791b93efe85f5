"""ORACLE — test infrastructure, not the product.

A plain, slow FP64 CPU implementation of the micromagnetic hot path of
arxiv 2608.15253 ("Claude-SpinDynamics"): finite-difference effective field
(exchange, interfacial and bulk DMI, uniaxial, cubic and surface
anisotropy, Zeeman, RKKY interlayer exchange, magnetoelastic field, Philox
thermal field, open and periodic (image-sum) Newell-tensor FFT
demagnetisation), the LLG right-hand side with spin-orbit / Slonczewski /
Zhang-Li torques, Heun, Dormand-Prince RK45, classical RK4 and the
Depondt-Mertens rotation scheme (fixed and adaptive), ensembles of trials
with retire/refill (``oracle.trials``), energy, topological charge and
mean magnetisation.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import it.  It shares no code with the CUDA path
(``paper_2608_15253_gb300``); both take their inputs from ``workloads``.

Every function cites the passage of the paper it follows (Methods,
"Physics and discretization", Eq. 1; "Integrators"; "Replica batching").
Where the paper is silent the reading taken is stated in the function.

Parity status: every function here is pinned by tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force, values
the paper prints, published known answers).  The surrogate network's
functions (``oracle.cnn``) are pinned as operations: the forward pass
against scipy's 2-D correlation, the gradients against finite differences
of the loss, the optimiser step and BF16 rounding by their definitions.
What a trained network predicts has no closed form; its error is measured
against the exact demagnetising field, not held to a parity bar.
"""
from .constants import MU0, GAMMA0, KB, HBAR, QE, MU_B  # noqa: F401
from .fields import (  # noqa: F401
    Problem, h_exchange, h_dmi, h_dmi_bulk, h_anisotropy, h_zeeman, h_cubic, h_surface, h_rkky,
    h_magnetoelastic, h_local, h_eff, neighbour_values,
)
from .demag import (  # noqa: F401
    newell_octant, newell_at, newell_analytic, newell_quadrature, newell_f, newell_g,
    newell_octant_images, padded_kernel, demag_spectrum, h_demag, h_demag_direct,
)
from .philox import philox4x32_10, splitmix64, uniforms, normals, thermal_field  # noqa: F401
from .llg import (  # noqa: F401
    Torque, llg_rhs, spin_torque, zhang_li_torque, rotate, Solver,
    DP_A, DP_B5, DP_B4, DP_C,
)
from .observables import energy, topological_charge, topological_charge_bl  # noqa: F401
