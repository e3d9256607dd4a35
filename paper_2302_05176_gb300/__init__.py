"""GB300-native k-register Gumbel-Max sketch (FastGM, arXiv 2302.05176).

The compute path is the CUDA library ``libgm`` (see ``include/gm.h``); the
Python binding in ``paper_2302_05176_gb300.gm`` only marshals arguments into
its C-ABI.  Importing this package does not load the library; the first call
through the binding does, and it raises if the library is missing.
"""
