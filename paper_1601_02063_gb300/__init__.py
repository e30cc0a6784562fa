"""GB300-native backward ray tracing and radiative transfer in Kerr spacetime.

The compute path lives in the CUDA library ``libodyssey_gb300.so`` (sources under
``csrc/``, C ABI declared in ``include/odyssey.h``); ``binding`` marshals arguments
to it.  Importing this package does not load the library.
"""
