"""GB300 (sm_103a) library for the time-domain SBFEM full-waveform-inversion hot path.

``paper_2501_06748_gb300.sbfwi`` is the Python binding of ``libsbfwi.so`` (C ABI in
``include/sbfwi.h``); ``paper_2501_06748_gb300.build`` compiles the library in-tree.
The binding is imported explicitly so that building does not need a built library.
"""
