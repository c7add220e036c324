"""GB300-native orthogonal-projector multigrid MLMC trace estimation.

The compute path is the C-ABI library ``libmgmlmc.so`` (CUDA for sm_103a),
reached through ``paper_2509_11424_gb300.mgmlmc`` (ctypes, argument marshalling
only).  ``synth`` holds the seeded input generators.
"""
