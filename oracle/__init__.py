"""FP64 CPU oracle for the implicit FFT elastodynamics method (arXiv 2211.08263).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA library: the only module both sides use is the seeded input generator
``paper_2211_08263_gb300.inputs``, which holds none of the method's arithmetic.

Modules:
  medium    -- voxel medium: per-voxel 4th-order stiffness tensors and density
  spectral  -- discrete frequencies, spectral derivatives, operator A, b,
               reference-medium preconditioner M (Sec. 2.2.2-2.2.3)
  pcg       -- masked preconditioned conjugate gradient, unmasked PCG
  newmark   -- beta-Newmark stepping with the prescribed-displacement region
  dense     -- dense differentiation matrices (closed form), dense A,
               constrained direct solve
  green     -- the paper's literal Green's-matrix Dirichlet method (Alg. 2)
  analytic  -- closed forms used as pins: plane waves, d'Alembert, wave speeds
  conv      -- FP64 3-D convolution network (learned warm start) fwd/bwd

Every function states the passage of the paper it follows.
"""
