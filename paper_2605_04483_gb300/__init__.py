"""GB300-native CDFCI column update (coordinate-descent FCI, CDFCI / mCDFCI).

The compute path is the CUDA library ``libcdfci.so`` behind the C-ABI declared
in ``include/cdfci.h``; ``paper_2605_04483_gb300.api`` is its thin Python
binding.  ``paper_2605_04483_gb300.inputs`` draws the seeded synthetic
workloads.  Nothing is imported eagerly here.
"""
