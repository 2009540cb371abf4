"""GB300-native P2S turbulence simulator (Mao, Chimitt & Chan, ICCV 2021).

The compute path lives in the C-ABI library libp2s (CUDA, sm_103a) built from
csrc/; `p2s` is its thin ctypes binding.  Importing the package does not load
the library; the first call into `p2s` does, and fails loudly if it is missing.
"""
