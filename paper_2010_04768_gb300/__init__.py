"""GB300-native GFCCSD hot path: shifted complex linear solves for the
Green's function G_pq(omega) (IP and EA sectors) behind a C ABI.

Importing the package loads nothing; ``paper_2010_04768_gb300.gfcc`` is the
ctypes binding to the CUDA library and ``paper_2010_04768_gb300.synthetic``
holds the seeded input generators.
"""
