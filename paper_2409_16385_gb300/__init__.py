"""GB300-native contact stage of Embedded IPC (arxiv 2409.16385).

The compute path is the CUDA library libembipc.so (C ABI in include/embipc.h, kernels in
csrc/, built by build.py for sm_103a); `binding` marshals torch CUDA tensors into it.
`scenes` builds the seeded synthetic inputs.  Above the contact stage: `elastic` and `sim`
(the reduced Newton driver), `adjoint` (autograd through the contact stage and through
trajectories), `autotune` (launch shapes)."""
from .binding import (BSR, ContactScene, LagState, PairList, accd_toi, bsr_spmv, build_candidates, eval_contact,
                      library_path, load, make_params)

__all__ = ["BSR", "ContactScene", "LagState", "PairList", "accd_toi", "bsr_spmv", "build_candidates", "eval_contact",
           "library_path", "load", "make_params"]
