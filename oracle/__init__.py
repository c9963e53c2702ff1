"""CPU FP64 oracle of the GFCCSD hot path.

Test infrastructure: only tests/, the smoke check and the bench's CPU-baseline
leg use this package.  It shares no code with the CUDA library; the seeded
input generators (paper_2010_04768_gb300.synthetic) are the only common module.
"""
