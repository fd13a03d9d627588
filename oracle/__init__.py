"""FP64 CPU oracle for the gauged superposition of Gaussian fermionic PEPS.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute anything under ``oracle/``; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and reference
legs) use it.  The oracle shares no code with the CUDA library: it has its own
Philox generator, Pfaffian, Fock-space machinery and weight formulas.

Modules
-------
philox   Philox4x64-10 counter generator (Salmon et al., SC'11).
         Groups: Z2, U(1) and SU(2) (doublets on the link ends; oracle only).
pfaffian Plain Parlett-Reid Pfaffian in C (complex and real FP64).
fock     Brute-force Fock-space construction and contraction of the PEPS
         (Sec. 3, Sec. 4, App. C): the definition of psi_n(G) written out.
weight   The covariance-matrix route of Sec. 5: Gamma_A(G) = O^T Gamma_A O,
         N_nm(G), <B_n|B_m> with the B_0 phase convention, N(G), p(G).
mcmc     Sequential-sweep Metropolis over link configurations (Sec. 5.1),
         full recomputation of N(G) for every proposal.
observables  Plaquette Wilson loops (Sec. 2.3) and integrated
         autocorrelation times.
electric The Z2 electric (link-flip) observable of Sec. 5.3: f_E(G) from
         explicit vectors and from a Pfaffian of the composed covariance.
fermionic  Majorana expectations of Sec. 5.2 (densities, link bilinears,
         general monomials, gauge-invariant link terms) from explicit
         vectors and from the physical covariance A + B W B^T of each pair.
variational  Per-configuration K x K matrices of the observables (Hermitian
         forms in lambda) and the generalised-eigenvector optimum of lambda.

Parity status per function is listed in each module's docstring; every
function is pinned by a `-m "not gpu"` test except where a docstring says
"parity unpinned".
"""
