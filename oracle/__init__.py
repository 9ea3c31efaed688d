"""Plain, slow FP64 CPU oracle for UNO-CG on periodic voxel homogenization problems.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.  It shares no
code with the CUDA path (no kernels, headers, tables or helpers); both sides only read the same
seeded inputs from the ``synth`` package.

Everything is float64 NumPy/SciPy written for readability, following the paper:

* ``fem``        Galerkin FE on a regular periodic voxel grid (Sec. 4.1, Eq. (fem-linear-system)),
                 thermal (Sec. 6.1) and linear-elastic (Sec. 6.2) homogenization problems.
* ``dft``        the unitary discrete Fourier transform written out by its definition.
* ``uno``        the UNO preconditioner P = T^H Q T (Eq. (FNOCG-prec-fields-disc)), the local
                 parametrization psi (Sec. 5.2.2, App. B.1) and the reference-medium
                 fundamental solution of FANS (Sec. 4.3.4).
* ``pcg``        preconditioned CG, Algorithm 1 / Algorithm 2, and a flexible variant.
* ``homogenize`` solves, effective tensors, sensitivities and a dense direct solve.
* ``training``   the MSE training loss of Eq. (fnocg-loss) and its gradients (Sec. 5.3, 5.4).
"""
