"""GB300-native Intergrams: top-k n-gram counting by multi-pass candidate scan.

The compute path is the native library ``libintergrams.so`` (sm_103a kernels
behind a C ABI); :mod:`.binding` marshals arguments to it. :mod:`.synth`
generates seeded synthetic corpora.
"""
__all__ = ["synth", "binding"]
