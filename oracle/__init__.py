"""Plain CPU oracle of the DPG ultraweak time-harmonic Maxwell method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2609_03155_b300``): its own bases,
quadrature, element formation, numbering, assembly, solvers and estimator,
written in complex FP64 numpy from the paper's statement of the method:

* Sec. 2.1, Eq. (final_dpg_formulation): the practical DPG mixed form.
* Sec. 2.2, Eqs. (maxwell_dimensionless), (bilinear_form), (trace_pairing),
  (linear_form), (test_inner_product): the ultraweak Maxwell forms and the
  adjoint graph test norm with alpha = 1.
* Sec. 2.3: the discrete spaces, the element block system, the two static
  condensations, Eq. (linear_system), local recovery and the residual
  estimator ||Psi||_V.
* Sec. 4.1: the TE_mn closed form and the port / impedance / PEC conditions.

Readings of the paper taken here (the paper is silent or ambiguous):

* Space indices (Sec. 2.3 vs Fig. 1 caption): interior DG degree p per
  component; trace = tangential trace of the Nedelec space of FEEC order p+1;
  test = Nedelec of FEEC order p+1+dp.  Pinned by the paper's DoF counts
  (Sec. 4.1: 720 on the coarsest waveguide level, about 1.65 M on the finest).
* The Robin term of Eq. (bilinear_form) acts on the trace E-hat (Algorithm 2
  puts the Robin contribution in (G, B-hat, l)).
* Psi = G^{-1}(l - B u - B-hat u-hat), the sign of the block system of Sec. 2.3
  (the printed recovery formula has the opposite sign; eta is unaffected).
* H-hat unknowns that pair with nothing (face DoFs on Robin faces, Sec. 2.3
  end) are removed from the global system.
* Dirichlet trace data is imposed by nodal interpolation of the tangential
  field at the Nedelec nodes.
* Mixed trial degrees (``mixed``): an edge or face carries trace unknowns of
  order min over its elements of p + 1; each element computes at its own
  degree and sees the global trace through nodal evaluation, u-hat_K = R_K u-hat.
* 2:1 hanging faces (``hanging``): an edge or face inside a larger neighbour
  entity takes that entity's trace (no unknowns of its own).
* Absorbed power and its adjoint gradient (``power``, ``adjoint``): Q_em of
  Sec. 3.2; the gradient with respect to Re eps and Im eps separately (G_K is
  not holomorphic in eps).

Functions whose result has no independent pin are marked "parity unpinned" in
their docstring; every other function is pinned by ``tests/test_oracle_*``.
"""
