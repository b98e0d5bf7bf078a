"""CPU oracle of the CCMF FFT-ADMM solver: test infrastructure only.

Only tests/, the smoke check and the CPU-baseline leg of bench.py may use it.
"""
