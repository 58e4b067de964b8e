"""GB300 (sm_103a) implementation of the frequency-domain secure convolution
(FDSC) hot path of ENSEI (Bian et al., CVPR 2020).

The compute lives in ``libfdsc.so`` (CUDA kernels behind the C ABI declared
in ``include/fdsc.h``); :mod:`paper_2003_05328_gb300.fdsc` is its Python
binding and :mod:`paper_2003_05328_gb300.build` compiles it.
"""
from . import fdsc  # noqa: F401
from .fdsc import (FdscError, LayerSpec, Params, decrypt, decrypt_share, encode_share, encrypt,  # noqa: F401
                   encrypt_constants, filter_prepare, homconv, homconv_sum, homrec, homrec_share, intt2d, keygen,
                   layout, mask_prepare, ntt2d, params_query)
