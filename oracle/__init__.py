"""FP64 CPU oracle of the GES render path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does; the two share no code.
"""
from .oracle import (DEFAULT_OPTS, build, load, render, backward, sh_basis, surfel_eval,
                     surfel_info, gauss_info, id_validity, touching,
                     count_fragments, filter3d, render_geom, render_translucent, backward_translucent,
                     covering_counts, contribution)

__all__ = ["DEFAULT_OPTS", "build", "load", "render", "backward", "sh_basis", "surfel_eval",
           "surfel_info", "gauss_info", "id_validity", "touching",
           "count_fragments", "filter3d", "render_geom", "render_translucent", "backward_translucent",
           "covering_counts", "contribution"]
