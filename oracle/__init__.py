"""FP64 CPU oracle for the SORF + FCHL19 approximate kernel method.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
restatement of what the method computes, written from the paper (Browning,
Faber, von Lilienfeld, "GPU-Accelerated Approximate Kernel Method for Quantum
Machine Learning"). Only the tests, the smoke check and the CPU-baseline leg
of the benchmark import it. The CUDA library never calls into it and shares no
code with it; both are fed the same seeded inputs from the synthetic
generators.

Modules
-------
fchl19      FCHL19 two- and three-body representation (Representation section,
            two-body, cutoff, three-body, ATM and Fourier-angular equations),
            in torch float64 so that forces and force rows come from
            automatic differentiation of the plain definition.
sorf        Walsh-Hadamard matrix by the Sylvester recursion, the dense SORF
            matrix W = (sqrt(d)/sigma) [H D_i]_{N_transform}, RFF, and the
            feature map z = sqrt(2/N_F) cos(W x + b) (RFF and SORF sections).
regression  per-element PCA basis (SVD projection equations), per-molecule
            feature matrix Z, regularised normal equations and their solve
            (normal-equation equations of the RFF section).
model       energies E = sum_I alpha^T z(rho_I), forces -dE/dr and the
            derivative-feature rows used for energy+force training.

Every routine works in float64. Parity is pinned by the tests under
``tests/test_oracle_*.py`` against closed forms, invariances, explicit
matrices, finite differences and library least squares.
"""
