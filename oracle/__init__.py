"""FP64 CPU oracle for the APIC augury contact step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does.
"""
from .oracle import (  # noqa: F401
    FLAG_PIC,
    FLAG_SEP23,
    build,
    weights,
    undesirable,
    D_tensor,
    p2g_grid,
    g2p_from_grid,
    apply_H,
    momentum,
    contact_step,
    apic1d_linear,
    node_normals,
    weight_grads,
    mass_normals,
    MASS_NORMAL_THRESHOLD,
    augury_steps,
)
