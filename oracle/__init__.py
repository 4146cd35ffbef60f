"""Plain FP64 CPU oracle for the MULTIBAT hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import anything from this package.  The product path
(the C-ABI library and its Python binding) never imports, links or calls it,
and this package imports nothing from the product package.

Modules
-------
fom   Full-order model: cell-centred finite-volume residual of the coupled
      electrolyte / solid / interface equations (Sec. 2.2-2.4, Eqs. cgr,
      phigr, cel, phiel, interfaceCond, ise_gr, ise_li, iplel and the
      implicit Euler system ap4:detailed), its Jacobian by complex-step
      differentiation, and a Newton step solved with SciPy's sparse direct LU.
rom   Reduced model: POD, EI-Greedy, Galerkin projection of the operator
      split and the fully reduced Newton solve (Sec. 2.5, Eqs. ap4:reduced,
      ap4:operator_decomposition, ap4:operator_subdecomposition,
      ap4:fully_reduced).

Parity status of each function is stated in its module header.
"""
