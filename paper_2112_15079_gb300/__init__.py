"""GB300-native direct-sum N-body with velocity Verlet (arXiv:2112.15079).

Submodules:

* ``inputs`` -- seeded synthetic Solar-System-shaped initial conditions
  (no force or integrator arithmetic; shared by tests, benchmark and oracle).
* ``nbody``  -- ctypes binding of the CUDA C-ABI library ``libnbody.so``.
  Importing it fails loudly when the library has not been built.
* ``autograd`` -- ``torch.autograd.Function`` over the adjoint entry point.

Nothing is imported eagerly, so the CPU-only parts stay importable on a
machine without the built library.
"""
__all__ = ["inputs", "nbody", "autograd"]
