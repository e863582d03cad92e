"""GB300-native batched nested slice sampling with fused emulator cosmic-shear
likelihoods (arXiv:2509.13307).

The numerical work lives in libgpuns.so (CUDA for sm_103a, C ABI in
include/gpuns.h); this package only marshals arguments.  Import is lazy: the
library is loaded on first use and its absence is an error, never a fallback.
"""

__all__ = ["Problem", "NestedRun", "MultiRun", "ShardedRun", "shard_bounds", "LogLike", "loglike_autograd", "nuts",
           "build"]


def __getattr__(name):
    if name in ("Problem", "NestedRun", "MultiRun", "ShardedRun", "shard_bounds", "LogLike", "loglike_autograd",
                "nuts"):
        from . import api
        return getattr(api, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
