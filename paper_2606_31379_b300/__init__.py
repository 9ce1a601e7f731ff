"""P3MaZe long-range electrostatics on one B300 (sm_103a).

The CUDA library and its ctypes binding live in ``paper_2606_31379_b300.p3maze``;
importing this package alone loads nothing.
"""
