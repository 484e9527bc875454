"""FP64 CPU oracle for QAOA Max-Cut expectation values and gradients.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path; the only
common dependency is the seeded input generator package ``synth``.

Parts (each module cites the passage it follows):

* ``statevector`` — O-SV: the plain definition, a 2^n complex128 state
  vector for the QAOA circuit of Section 4.1, with <Z_a Z_b>, <C>, amplitudes
  and an adjoint-method gradient.
* ``lightcone``  — O-LC: the same state vector restricted to the radius-p
  ball around an edge (exact for <Z_u Z_v>).
* ``tensornet``  — O-TN: the ket/bra tensor network of the circuit,
  contracted by plain variable elimination (Eq. 1 as numpy einsum) in a
  greedy min-degree order; gradient by forward-mode dual tensors.
* ``closed_form`` — the known p=1 closed form of <Z_u Z_v> and its
  derivatives.
* ``superop``    — the paper's dim-4 superoperator tensors (Section 2) and
  a density-matrix network evaluator, used to pin the bond-dimension-2
  sandwich reading against the paper's own form.
* ``answer``     — Section 3.3's sequential answer-string estimate over an
  exact probability vector.
* ``density``    — O-DM: the density matrix of the QAOA circuit with a
  Kraus channel (depolarizing, dephasing, amplitude damping) on every qubit
  after each layer's mixer; <Z_a Z_b>, <C> and a finite-difference gradient.

Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (scipy's matrix exponential, the closed form, invariants,
finite differences, brute force); no function is "parity unpinned".
"""
