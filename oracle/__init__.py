"""CPU FP64 oracle for the binned-FFT bandwidth-selector functionals.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) use it.  It shares no code, tables or constants with
the CUDA library; both sides receive the same seeded inputs from
``paper_1511_07482_gb300.synthetic``, which holds none of the method's
arithmetic.

Paper: Gramacki & Gramacki, "FFT-Based Fast Bandwidth Selector for
Multivariate Kernel Density Estimation" (arXiv 1511.07482).  Citations below
use the paper's own numbering: Sec. 3 (bandwidth selectors), Sec. 4 (the
four-step FFT algorithm), Sec. 5 (integrated density-derivative functionals),
Eqs. 8-36, Tables 2-3.

Modules
  gauss       Gaussian density derivatives via the multivariate Hermite
              recurrence (the D^{(x)r} phi_Sigma of Sec. 5, Eqs. 13, 30-31).
  rules       bin width (Eq. 16), effective support L_k (Eq. 26), padded
              sizes P_k (Eqs. 21, 27 and the minimal no-alias reading).
  binning     linear and simple binning (Sec. 4, first step).
  functionals direct double sums (Eqs. 12-13, 29), binned double sum
              (Eq. 25) and the paper's four FFT steps (Eqs. 17-24).
  selectors   LSCV (Eqs. 8, 10-11), SCV and plug-in objectives (readings of
              the Sec. 5 closing remark), psi_r vectors, analytic gradients.

Parity status of each function is stated in its docstring; the SCV and PI
formulas are readings of sources the paper cites but does not print, so
their *formulas* are pinned only to closed forms and identities, not to the
paper.
"""
