"""FP64 CPU oracle for the circuit / density-matrix hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct restatement of what the thesis defines (state vectors, gates,
quantum operations, Pauli transfer matrices, the Born rule).  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it;
the library never does, and it shares no code with the CUDA path.

Modules
-------
gates        gate matrices: rotations (Eqs. (singlequbitrotationx-z)), U1-U3
             (Eqs. (singlequbitU1-U3)), Tab. (elementarygateset), CNOT
             (Eq. (cnotgate)), CZ, CP.
statevector  gate application on bit positions, full 2^n x 2^n products,
             probabilities (Born rule), QFT closed form (Eq. (multiqubitqft)).
density      density matrices, unitary maps and Kraus channels (Sec. "Quantum operations"),
             Pauli basis, Pauli transfer matrices (Eq. (paulitransfermatrix)),
             Pauli vectors (Eqs. (GSTVectorizedRho), (GSTVectorizedEJ)),
             depolarizing and amplitude-damping channels
             (Eqs. (singletDepolarizingChannel),
             (singletAmplitudeDampingChannel1-2)).
noisy        the batched noisy-circuit forward model, multinomial
             log-likelihood and its gradient (finite differences and an
             independent adjoint in the density-matrix picture).
gradient     state-vector adjoint / finite-difference parameter gradients.
readout      the measurement-error model (Eq. (errordetectionMeasurementError))
             and the Bloch vectors of every qubit (Eq. (multiqubitblochvector)).
gst          GST predictions for repeated gates (Eq. (GSTPrediction)) and the
             statistical distance (Eq. (statisticaldistance)).
code422      the [[4,2,2]] error-detection experiment: bare and encoded circuits
             (Tabs. (errordetectionstates), (errordetectiongates)), postselection
             and D_bare/enc (Eq. (errordetectionDbareenc)).

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, printed values of the thesis and brute force.
"""
