"""GB300-native (sm_103a) FP64 particle tracker: the data-parallel hot path of
GPU-accelerated Elegant (arXiv:1710.07350) behind the C ABI of include/trk.h.

The Python binding (``paper_1710_07350_gb300.trk``) only marshals arguments;
all tracking runs in the CUDA kernels of libtrk.so.
"""
