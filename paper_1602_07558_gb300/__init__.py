"""GB300-native swept rule for explicit time advancing of 2D PDEs on periodic grids.

The compute path is the C-ABI library ``libswept2d.so`` (hand-written CUDA for
sm_103a, sources in ``csrc/``, declarations in ``include/swept2d.h``); the
Python binding ``swept2d`` only marshals arguments into it.
"""
