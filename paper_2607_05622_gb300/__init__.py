"""GB300-native Laplace-transform AO-direct J/K build and its gradient adjoint.

The CUDA library is loaded lazily by ``paper_2607_05622_gb300.ltjk``; importing
this package alone loads nothing.
"""
