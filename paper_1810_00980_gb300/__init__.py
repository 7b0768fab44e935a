"""GB300-native delta-temporal motif counting and the interval-sampling
estimator of Liu, Benson & Charikar (WSDM 2019).

The compute path is the CUDA library ``libtmotif.so`` (C ABI declared in
``include/tm.h``); ``paper_1810_00980_gb300.tm`` is its thin Python binding.
``paper_1810_00980_gb300.synth`` draws seeded synthetic temporal graphs.
"""
__all__ = ["tm", "synth"]
