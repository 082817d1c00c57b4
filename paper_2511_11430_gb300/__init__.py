"""GB300-native vortex-particle hot path of the NL-UVLM-VPM method (arXiv 2511.11430).

``api`` wraps the C ABI of include/vpm.h for CUDA tensors, ``autograd`` exposes the
adjoint as a torch.autograd.Function, ``synth`` builds the seeded synthetic rotor
wakes, and ``build`` compiles libvpm.so for sm_103a.  Importing the package does not
load the CUDA library; the first call into ``api`` does, and fails loudly if it has
not been built.
"""

__all__ = ["api", "autograd", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
