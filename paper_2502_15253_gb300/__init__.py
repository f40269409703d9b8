"""GB300-native forward-folding likelihood fits (PhyLiNO, arXiv 2502.15253).

Submodules:
  synth     - seeded synthetic model descriptions, ensembles and pseudo-data (inputs only)
  fitcore   - ctypes binding of the C ABI of libfitcore.so (include/fitcore.h)
  ensemble  - checkpointed ensemble fits and their JSON-lines output (host orchestration)
  warmstart - the warm-start network's argument tables and weight files
  cli       - command line: configuration in, fits on the GPU, JSON records out
  build     - nvcc build of libfitcore.so for sm_103a
"""
__all__ = ["synth", "fitcore", "ensemble", "warmstart", "cli", "build"]
