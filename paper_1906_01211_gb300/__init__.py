"""GB300-native AMOEBA induced-dipole polarization solve.

Submodules:
  amoebapol  ctypes binding of the C-ABI library libamoebapol.so (solve,
             energies, forces, list reuse, predictor, permanent multipoles)
  torch_api  torch.autograd functions of the polarization and multipole energies
  serve      continuous-batching server of solve requests over CUDA streams
  synth      seeded synthetic water systems (inputs only)
  build      nvcc build of libamoebapol.so for sm_103a
"""
__version__ = "0.1.0"
