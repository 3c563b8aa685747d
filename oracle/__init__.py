"""FP64 CPU oracle for the differentiable cosmological hydro step (arXiv 2502.02294, diffHydro).

This package is TEST INFRASTRUCTURE. It is a plain, slow, float64 restatement of what the
paper computes, written with PyTorch CPU tensor operations so that ``torch.autograd`` gives
the exact reverse-mode gradient of the same arithmetic (the paper differentiates its JAX
simulator the same way, Sec. 2.3.5). Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The product path
(the CUDA library and its Python binding) never imports, links or executes anything here,
and nothing here imports the product.

Modules and the passages they follow:

* ``cosmology``  -- background E(a), linear growth D(a), FastPM kick/drift factors (Sec. 2.2).
* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al. 2011), the uniform
                    and Gumbel(0,1) draws of Sec. 2.4.2 and Box-Muller normals for the ICs.
* ``hydro``      -- relaxing TVD sweep (Sec. 2.3.1-2.3.2, Eqs. TVD_halfstep / TVD_fullstep,
                    van Leer limiter) and the Strang permutation cycle.
* ``pm``         -- CIC deposit / readout, spectral Poisson force, kicks and drift (Sec. 2.2,
                    Eqs. dm_hamil, the gravity source S_g of Eq. conservation).
* ``subgrid``    -- star formation with sigmoid thresholds and Gumbel-softmax relaxation
                    (Sec. 2.4.1-2.4.2, Eqs. reparam / gumbelsoftmax, pi_0(rho, T)).
* ``ics``        -- Gaussian realisation and Zel'dovich displacement of DM and gas (Sec. 2.1).
* ``spectra``    -- binned power spectrum and cross-correlation coefficient r_c (Sec. 3.1, 3.2).
* ``sim``        -- one full time step and a run, parameters, losses.
* ``closure``    -- the learned per-step correction (Sec. 4, solver-in-the-loop): periodic
                    3x3x3 convolutions with GELU in bfloat16-quantised float64, its loss and
                    Adam update, and the coarse/fine pairing operators of its training runs.

Every function here is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, textbook solutions, published constants, invariants, finite
differences). Functions without such a pin say "parity unpinned" in their docstring.
"""
