"""GB300-native (sm_103a) DEM hot path of the adaptive coarse-grain method
(Queteschiner et al., 2017): cell-list neighbour search, damped Hertzian
contacts with tangential history and Coulomb truncation, velocity Verlet.

The compute path is the C-ABI library ``libcgdem.so`` built from ``csrc/``;
``paper_1705_03850_gb300.dem`` is its thin ctypes binding.
"""
__all__ = ["dem", "workloads"]
