"""GB300-native contact stage of Embedded IPC (arxiv 2409.16385).

The compute path is the CUDA library libembipc.so (C ABI in include/embipc.h, kernels in
csrc/, built by build.py for sm_103a); `binding` marshals torch CUDA tensors into it.
`scenes` builds the seeded synthetic inputs."""
from .binding import (BSR, ContactScene, LagState, PairList, accd_toi, build_candidates, eval_contact,
                      library_path, load, make_params)

__all__ = ["BSR", "ContactScene", "LagState", "PairList", "accd_toi", "build_candidates", "eval_contact",
           "library_path", "load", "make_params"]
