"""FP64 CPU oracle of the differentiable direct-sum N-body method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product package never
imports it; the two share no code.

Modules:
  core    -- ctypes wrapper of the C oracle (pair gravity, NFW / Miyamoto-Nagai
             potentials, kick-drift-kick integrator, discrete adjoint).
  stream  -- the stream-density head (projection to (phi1, phi2), soft 2-D
             histogram, squared-error loss) and its adjoint, plus the whole
             mock-stream pipeline of Fig. 2 and its gradient.
  mlp     -- FP64 reference of the density surrogate network and Adam.
"""
from . import core  # noqa: F401
