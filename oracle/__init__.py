"""CPU oracle of the thermal pseudopotential D3Q19 lattice Boltzmann method (FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline leg. It shares no code with the CUDA path and never imports it.
"""
