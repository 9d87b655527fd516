"""FP64 CPU oracle for the sliced pairwise contraction of quantum-circuit tensor
networks.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
benchmark's timed CPU baseline may import it; the library's compute path never
does, and the two share no code (both only read the seeded inputs built by
the `circuits` package).

Three independent routes to the same numbers:
  * statevector  (O1): dense FP64 state vector, gates applied in circuit order
                        (Section 2.2), plus the adjoint sweep for gate environments.
  * einsum       (O2): the tensor network contracted pairwise (Section 2.3,
                        Eq. sequence) with numpy.tensordot as the pairwise step;
                        slicing by fixing index values (Section 2.4, Eq. sliced_sum);
                        bras attached as literal rank-1 tensors (Section 2.2.1).
  * sector       (O1 for bosonic networks): the same state vector restricted to
                        one total-photon sector (beamsplitters conserve the photon
                        number), so 16-mode, d = 4 lattices fit a host.
  * naive        (A3): the literal sum over every index assignment of the product
                        of all tensor entries (Eq. naive_summation), tiny cases only.
Every function here is pinned by tests against closed forms, brute force and
the paper's worked example rather than against itself.
"""
from .statevector import sv_state, sv_amplitudes, sv_env, gate_arrays
from .einsum import (contract_network, greedy_path, attach_bras, slice_network,
                     amplitude, sliced_partials, network_flops)
from .naive import naive_sum
from .sector import sector_amplitudes, sector_dim

__all__ = ["sv_state", "sv_amplitudes", "sv_env", "gate_arrays", "contract_network",
           "greedy_path", "attach_bras", "slice_network", "amplitude", "sliced_partials",
           "network_flops", "naive_sum", "sector_amplitudes", "sector_dim"]
