"""GB300-native FCC cosine transform (Seifert, Hueper, Uhl 2018).

The compute path is the CUDA library ``libfccdct.so`` behind the C ABI in
``include/fcc_dct.h``; ``binding`` marshals arguments to it and nothing else.
Import of this package does not load the library: ``binding.lib()`` does,
and raises if the library is missing (there is no CPU fallback).
"""
