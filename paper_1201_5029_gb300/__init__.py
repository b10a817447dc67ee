"""GB300-native symplectic lattice stepper (PyCOOL method, arXiv:1201.5029)."""
