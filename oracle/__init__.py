"""CPU oracle for the preconditioned nonlinear conjugate gradient (NCG)
micromagnetic minimiser (Exl et al., arXiv:1801.03690).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement
of the paper's method (Sec. 2.1-2.2, Algorithms 1 and 4, Eqs. energy, proj,
opt2, precond, t1-t3, li1-li3) written with numpy/scipy.  It shares no code
with the CUDA library and must only be imported by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.
The product path never calls it.

Units (a reading: the paper does not state them, but the stopping rules
t1-t3 compare energies against 1): lengths in nm, magnetisation in units of
M_ref = max Ms, energies in units of mu0*M_ref^2*(1 nm)^3, fields as
H / M_ref.  See ``fem.Units``.

Modules:
  fem         -- P1 tetrahedral assembly of C_A, C_K, the Ms weights, the
                 scalar-potential stiffness and the divergence coupling.
  linear_cg   -- Algorithm 1 (preconditioned linear CG).
  energy      -- magnetostatic potential, energy (Eq. energy), gradient,
                 projection (Eq. proj), normalised-objective derivative (Eq. opt2).
  precond     -- the sparse approximate Hessian (Eq. precond) and its
                 truncated inner solve (Algorithm 1 with li1-li3).
  ncg         -- Algorithm 4 with beta*ZA, the descent safeguard, the line
                 search and the stopping rules t1-t3.
  curve       -- the field sweep (demagnetisation curve) and coercive field.

Parity status: every function above is pinned by the not-gpu tests in
tests/test_oracle_*.py (closed forms, invariants, brute force, finite
differences); see each module's header.
"""
