"""FP64 CPU oracle for one Chebyshev-filtered subspace iteration (ChFSI) pass.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it; the only module both sides use is
``synth`` (seeded random numbers and analytic model functions).

It is a plain, slow, obviously-correct restatement of the paper's method
(DFT-FE 1.0, Das et al., Comput. Phys. Commun.), section by section:

  basis.py        GLL nodes/weights, Gauss rule, 1D Lagrange tables   (Sec. 2.3, Eq. fem; Eq. hep)
  mesh.py         periodic hexahedral spectral-element mesh, lumped M (Sec. 2.3)
  hamiltonian.py  cell matrices H~^c = M^-1/2 (K^c + V^c) M^-1/2,
                  H~X by gather / cell GEMM / assembly,               (Eq. discreteHam, Eq. hep,
                  nonlocal C~ h C~^T X                                 Eq. quadLocal/gemmLoc, Eq. celldgemm,
                                                                       Eq. nonlocalHamDiscrete, Alg. 4)
  chfsi.py        Chebyshev filter, Lanczos bounds, Cholesky-Gram-     (Eq. chebyfilter, Alg. 2)
                  Schmidt, Rayleigh-Ritz, residuals, one pass
  density.py      spectrum-splitting Rayleigh-Ritz, Fermi level,      (Alg. 2 step 3a, Alg. 3)
                  electron density at quadrature points
  mlp.py          the learned degree/bounds proposer's network:        (no counterpart in the paper)
                  forward, loss gradient by the chain rule, Adam
  kpoint.py       Bloch k-point Hamiltonian H~^k (complex cell terms    (Sec. 2, Eq. bloch and the
                  -i k.G^c + 1/2|k|^2 M^c, phased projectors) and the    reduced equation after it)
                  complex CholGS / Rayleigh-Ritz / residuals / pass

Every function is FP64.  Library primitives used as single steps: numpy
matmul/einsum, numpy.linalg.cholesky/eigh, scipy triangular solve, scipy.sparse
selection matrices for gather/assembly.

Pins (tests/test_oracle_*.py) tie it to closed forms and invariants: GLL p=4
closed form, quadrature exactness, Kronecker-sum spectrum of the free-electron
operator, harmonic-oscillator levels, scalar Chebyshev identity on exact
eigenvectors, nonlocal PSD/rank/normalisation, Courant-Fischer, convergence to a
dense eigensolve; for mlp.py, central finite differences, a closed-form linear special
case and Adam's closed-form first step; for kpoint.py, the Kronecker sum of 1D Bloch
operators, the free-electron closed form 1/2|k+G|^2 and Bloch folding of a doubled
supercell.  No function here is "parity unpinned".
"""
from .basis import gll_rule, gauss_rule, lagrange_table, lagrange_deriv_table
from .mesh import PeriodicMesh
from .hamiltonian import Hamiltonian
from .chfsi import (chebyshev_filter, lanczos_bounds, cholgs, rayleigh_ritz,
                    residuals, chfsi_pass, first_pass_bounds, Bounds)
from .density import (fermi_dirac, fermi_level, rayleigh_ritz_split, density, KB_HA_PER_K)
