"""CPU oracle for biorthonormal CCSD derivative couplings (test infrastructure).

Plain, slow, FP64 restatement of what the method computes.  Only the test
suite, the package's smoke check and the CPU-baseline leg of the benchmark
may import it; the CUDA library never links or calls anything here, and the
two share no code.

Modules
-------
fockspace : literal determinant-space evaluation of the paper's definitions
            (similarity-transformed Hamiltonian by matrix exponentials, the
            biorthonormal projection manifold, commutators) for tiny systems.
ccsd      : closed-shell CCSD residual and energy over Cholesky-factored
            integrals in T1-transformed form, plus the Jacobian, its
            transpose, the F-matrix and the Hamiltonian derivatives obtained
            by differentiating that residual (the Jacobian is the derivative
            of the residual with respect to the amplitudes).
solvers   : ground-state amplitudes, ground-state multipliers, EOM left/right
            states, biorthonormalisation, the coupling multipliers and the
            derivative coupling of Eq. (NAC_NC), plus a finite-difference
            evaluation of the definition Eq. (nac); state-energy gradients
            from the energy Lagrangian and finite differences of E_k(x).
relaxed   : Hartree-Fock orbitals, the orbital-response multipliers and the
            relaxed coupling.
meci      : the crossing-point search the couplings serve (branching plane
            from the energy-difference gradient and the coupling,
            Bearpark-Robb-Schlegel direction) on a synthetic family, from the
            CC oracle or from full CI.
mlp       : the learned doubles guess (features, network, gradients of its
            training loss), an extension outside the paper's method.
"""
