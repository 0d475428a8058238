"""GB300-native thermoelastic solver: P1/P2 assembly and SA-AMG-PCG in CUDA.

The compute path is the shared library ``libthermoamg.so`` (C ABI declared in
``include/thermoamg.h``); ``paper_1804_10060_gb300.thermoamg`` is its thin
Python binding.  ``meshgen`` makes seeded synthetic inputs.  Importing this
package does not load the library; importing ``thermoamg`` does, and fails
loudly when it has not been built.
"""
