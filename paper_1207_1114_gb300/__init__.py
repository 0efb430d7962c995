"""GB300-native FastPFP: projected fixed-point graph matching on sm_103a.

The solver lives in the C-ABI shared library built from ``csrc/`` (see
``include/fastpfp.h``); :mod:`paper_1207_1114_gb300.fastpfp` is the thin
ctypes binding with the same entry-point names.  :mod:`.synth` draws the
seeded synthetic inputs.
"""
