"""GB300-native AMOEBA induced-dipole polarization solve.

Submodules:
  synth      seeded synthetic water systems (inputs only)
  amoebapol  ctypes binding of the C-ABI library libamoebapol.so
"""
__version__ = "0.1.0"
