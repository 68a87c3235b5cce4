"""GB300 (sm_103a) dynamical-core library: Python side.

`paper_2511_02021_gb300.capi` is the ctypes binding of include/icon.h (same names
as the C entry points); importing it fails loudly if the CUDA library has not been
built (`paper_2511_02021_gb300.build.build()`). `use_torch_allocator` and
`bind_torch_stream` hand device memory and streams to the library from PyTorch,
which is used for nothing else.
"""


def use_torch_allocator(device=0):
    """Route every device allocation of the library through PyTorch's caching allocator."""
    import torch
    from . import capi
    stream = torch.cuda.current_stream(device)

    def alloc(nbytes):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        except Exception:          # out of memory: the library sees NULL and reports ICON_ENOMEM
            return 0

    def dealloc(ptr):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    capi.icon_set_allocator(alloc, dealloc)


def bind_torch_stream(stream=None):
    """Enqueue the library's work on a torch CUDA stream (default: the current stream)."""
    import torch
    from . import capi
    s = stream if stream is not None else torch.cuda.current_stream()
    capi.icon_set_stream(s.cuda_stream)
