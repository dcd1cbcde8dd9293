"""Named workloads shaped like the paper's experiments (Sec. 3): scan
geometry, batch, noise and phantom parameters, and the arithmetic each is
run in.  Host-side data only; `geometry(name)` turns one into the
ct_geometry the library takes.

The paper reconstructs real CT slices (Sec. 3.1, 3.2) with a fan-beam
scanner; these parallel-beam workloads keep its shape (a tall system matrix,
many slices per geometry, attenuation-like images with air around the
object, low-dose Poisson noise) at sizes from a 32 x 32 check up to the
512 x 512 image of the paper, and add the sqrt(lambda) I rows that keep the
regularised systems full rank.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    n_side: int           # image n_side x n_side, n = n_side^2 unknowns
    n_views: int          # views evenly over 180 degrees (endpoint excluded)
    n_bins: int           # detector bins of one pixel width
    sqrt_lambda: float    # 0: no regularisation rows
    slices: int           # sinograms per geometry
    i0: float | None      # incident photons per ray; None: noiseless data
    ellipses: int         # ellipses per phantom
    precisions: tuple     # arithmetic the workload is run in
    batch: int = 0        # slices per solve call (0: all at once)
    out_of_core: bool = False
    note: str = ""

    @property
    def n(self) -> int:
        return self.n_side * self.n_side

    @property
    def m(self) -> int:
        return self.n_views * self.n_bins

    @property
    def rows(self) -> int:
        """M' = m + n with regularisation rows, else m."""
        return self.m + (self.n if self.sqrt_lambda > 0 else 0)


PRESETS = {w.name: w for w in (
    Workload("plain_32", 32, 60, 46, 0.0, 1, None, 8, ("fp64", "fp32"),
             note="dense Householder QR and one solve of noiseless data; exact recovery"),
    Workload("plain_128", 128, 180, 182, 0.05, 64, 1e4, 10, ("fp32", "fp64"),
             note="FP32 against FP64 QR on the GPU, log-transformed Poisson data"),
    Workload("mixed_256", 256, 360, 364, 0.05, 512, 5e3, 10, ("tf32", "bf16"),
             note="tensor-core trailing updates with FP32 accumulation, FP64 refinement, "
                  "all slices in one solve"),
    Workload("diff_128", 128, 180, 182, 0.05, 256, 1e4, 10, ("tf32",),
             note="the autograd solve layer: loss = MSE to the phantoms, backward = the adjoint"),
    Workload("ooc_512", 512, 720, 730, 0.05, 1024, 1e4, 10, ("tf32", "bf16"), batch=256,
             out_of_core=True,
             note="matrix in pinned host memory or a file, factored in superpanels under a "
                  "device budget; slices solved in batches"),
)}


def geometry(name: str):
    """The library's parallel-beam ct_geometry of a preset."""
    from . import make_geometry
    w = PRESETS[name]
    return make_geometry(w.n_side, w.n_views, w.n_bins, w.sqrt_lambda)
