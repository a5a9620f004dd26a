"""FP64 CPU oracle and closed-form theory for the fluctuating Shan-Chen D2Q9
lattice Boltzmann method (arXiv:2212.07848).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the package smoke
check and by the benchmark's CPU-baseline leg, never by the product path.
It shares no code with the CUDA library.
"""
