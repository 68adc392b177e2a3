"""FP64 CPU oracle for the preconditioned primal-dual (PPD) imaging solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of what the method computes (Onose, Dabbech & Wiaux
2017, "An accelerated splitting algorithm for radio-interferometric imaging").
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls, links or shares
code with it; the two are fed the same inputs by
``paper_1701_01748_gb300.synth`` and compared.

Modules
-------
nufft  : Phi = Theta G F Z, its adjoint, the exact NUDFT, binning and the
         uniform-weighting preconditioner (Section 2, Section 5).
sara   : Daubechies filters and the SARA dictionary Psi / Psi^dagger
         (Section 2.2, Section 5.1).
prox   : proximity operators and the ellipsoid projection (Section 3.3,
         Section 4.1, Algorithm 2).
ppd    : parameters and one iteration of Algorithm 3 (Section 4).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against a closed form, a brute-force definition, an invariant or a special
case, except the full PPD trajectory beyond those invariants, which is
"parity unpinned" (it is pinned only through the invariants listed in
``oracle/ppd.py``).
"""
