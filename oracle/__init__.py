"""FP64 CPU oracle of the TCNS scheme (arXiv 1810.07806).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library
is checked against.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA path.
"""
