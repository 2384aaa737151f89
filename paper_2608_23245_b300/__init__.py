"""B300-native fiber-diffraction hot path (structure factors, shell-quadrature
profiles, Lorentz-corrected Ewald projection) behind the ``libfdx`` C-ABI.

The binding in :mod:`paper_2608_23245_b300.fdx` loads the CUDA library on first
use; importing the package itself loads nothing.
"""
