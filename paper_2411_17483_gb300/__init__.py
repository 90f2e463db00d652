"""SOFA exact k-NN over z-normalised data series, GB300 (sm_103a) native.

The compute lives in libsofa.so (C ABI: include/sofa.h); `sofa` is its
ctypes binding, `datagen` the seeded synthetic workload generators and
`shards` the host-side merge of per-shard k-NN windows.
"""
__all__ = ["sofa", "datagen", "shards"]
