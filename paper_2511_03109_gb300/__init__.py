"""GB300-native online stage of parametric H / H^2 kernel matrices.

The compute path lives in the C-ABI library ``libph`` (CUDA for sm_103a, built
by ``__graft_entry__.build()``); ``paper_2511_03109_gb300.ph`` is its thin
ctypes binding.  ``paper_2511_03109_gb300.inputs`` holds the seeded synthetic
workloads.  Importing this package does not load the library; importing
``paper_2511_03109_gb300.ph`` does, and fails loudly if it is missing.
"""
