"""GB300-native hyper-reduced (POD + ECM) RVE solver for the geometrically
parameterised elasto-plastic micro problem of arXiv 2307.16894.

Modules: ``binding`` (ctypes binding of the C ABI in include/podecm.h),
``build`` (nvcc build of libpodecm.so), ``workload`` (model files and batch
inputs), ``inputs`` (seeded synthetic input generators).
"""
