"""CPU oracle for the THC second-order-exchange (SOX / SOSEX) self-energy.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

Everything here is plain numpy (complex128 by default, float64 allowed for
real molecular data) written from the paper's definitions:

* ``grid``       Chebyshev-Lobatto tau grid, Clenshaw-Curtis weights, the
                 fermionic reflection G(-tau) = -G(beta - tau).
* ``thc``        THC factorisation (Sec. II C) and the projections of G onto
                 THC points.
* ``sox``        the SOX self-energy of Eq. (sox) with static interactions, by
                 three routes: brute force over the reconstructed 4-index
                 integrals, the pure-THC O(N^4) form, and the paper's chain
                 (Eq. U_contraction onward, Sec. II C).
* ``screening``  Pi(0) and W(i Omega = 0) for statically screened SOSEX.
* ``phi``        the Luttinger-Ward functional Phi_SOX and its gradients.
* ``dynamic``    dynamically screened SOSEX (Eq. GG onward, Sec. II C).
* ``kpoints``    the momentum-resolved forms for periodic solids.
* ``scloop``     the self-consistent loop around Sigma for molecules (Dyson equation
                 on fermionic Matsubara frequencies, chemical potential, Galitskii-Migdal
                 energies, Sec. II A).
"""
from . import grid, thc, sox, screening, phi, kpoints, dynamic, scloop  # noqa: F401
