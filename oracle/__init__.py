"""FP64 CPU oracle for the stresslet-constrained positively-split Ewald (PSE) method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs
this code; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg / ``--impl reference`` arm of ``bench.py`` may use it.

The oracle is plain and slow on purpose.  It follows the paper
(Fiore & Swan, "Rapid Sampling of Stochastic Displacements in Brownian Dynamics
Simulations with Stresslet Constraints", arXiv:1709.06946) step by step:

* ``params``     -- parameter rules (Sec. 2.3.1 real-space cutoff; Eq. bound with
                    m = sqrt(pi P); readings for k_cut and the grid size where the paper is silent).
* ``basis``      -- orthonormal symmetric-traceless basis for the 5 stresslet
                    components (Sec. 2.2.1 rigid-particle relation).
* ``realspace``  -- real-space split mobility M^(r) (Eqs. MUFr-MDCr, defined as
                    the inverse Fourier transform of M - M^(w)), evaluated as 3D
                    convolutions of sphere-shell / ball densities with the
                    split Hasimoto Green's function.
* ``wavesum``    -- direct wave-space k-sum of M^(w) (Eqs. MUFw-MDCw).
* ``ewald``      -- dense classical Ewald grand mobility (8N x 8N) for small N.
* ``pse``        -- the PSE algorithm (Sec. 2.3: spread, FFT, scale, iFFT,
                    interpolate; real-space pair sum; Sec. 3: split sampling with
                    Lanczos + wave-space noise; mid-point constrained step).
* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                    + Box-Muller, used where noise is drawn in-kernel.

Parity status of every function is stated in its module header.
"""
