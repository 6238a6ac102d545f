"""GB300-native adaptive Genz-Malik quadrature (arXiv 2511.01573 hot path).

``gmq`` is the binding of the CUDA library (C ABI in ``include/gmq.h``);
``genz_inputs`` draws the seeded synthetic test-family parameters.
"""
