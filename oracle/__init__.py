"""CPU FP64 oracle for the electrostatic Vlasov-Poisson PIC loop (Landau damping).

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously-correct
restatement of what the GPU library computes, written from the paper's
statement of the problem (Sec. 2, Eqs. 1-4; Sec. 2.1; Sec. 3.2) and from the
standard published methods named in each function. Only the test-suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it. The GPU library never calls it and it never
calls the GPU library: the two share no code, headers, tables or constants.

Modules
-------
philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11).
pic      Landau initial condition, CIC scatter, 7-point FD operator,
         Jacobi-PCG, discrete spectral solve, gradient, CIC gather,
         leapfrog push, field energy, and the full PIC loop.
cnn      3x3x3 conv3d forward/backward by direct loops, the 4-layer CNN
         preconditioner, its loss, Adam, and flexible CG (FCG(1)).
mg       geometric multigrid V-cycle preconditioner (textbook, beyond the
         paper): transfers, damped Jacobi, the cycle.
fft      FFT pseudo-spectral periodic Poisson solve (Sec. 3.1): phi and E.
ssor     red-black SSOR preconditioner (the paper's PCG configuration,
         Sec. 4.1).
pif      particle-in-Fourier field by direct non-uniform DFT sums (Sec. 3.4,
         Appendix A).
"""
