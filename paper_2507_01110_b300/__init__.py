"""B300-native LoD Gaussian splatting render path ("A LoD of Gaussians", arxiv 2507.01110).

The compute path is liblodgs.so (hand-written sm_103a CUDA behind a C ABI,
include/lodgs.h).  `api` is its Python binding, `autograd` the
torch.autograd.Function around render/render_backward, `serving` the
continuous-batching request loop, `synth` the seeded synthetic inputs.
Submodules are imported lazily so that importing the package needs no GPU.
"""
__all__ = ["api", "synth", "build"]
