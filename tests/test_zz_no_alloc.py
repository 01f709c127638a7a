"""pic_read_emag_noalloc against pic_read_fields(PIC_FIELD_EMAG).

The no-allocation read-out serves callers that cannot call cudaMalloc (for example code
running while another thread captures a CUDA graph, or callers whose device memory belongs to
an outside allocator).  It must give the same |E| per leaf as the allocating read-out, call
after call, and refuse meshes beyond its fixed 131,072-leaf scratch.  This file is collected
last so that a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process (the first call does the per-device set-up).
"""
import numpy as np
import pytest

import paper_1604_07713_gb300 as G
from paper_1604_07713_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx_with_fields(precision):
    tree = W.streamer_tree(nx0=32, lmax=3)
    cfg, mesh, parts = W.streamer(n_particles=20000, nx0=32, lmax=3, precision=precision, tree=tree)
    ctx = G.Context(cfg)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        ctx.load(s, **parts[s])
    ctx.compute_fields()
    return ctx


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
def test_noalloc_emag_matches_allocating_readout_twice(precision):
    G.build()
    with _ctx_with_fields(precision) as ctx:
        ref = ctx.fields(G.PIC_FIELD_EMAG)
        assert ref.size > 1000 and np.abs(ref).max() > 0
        for _ in range(2):  # two calls in a row share the fixed scratch
            out = np.full(ref.size, np.nan)
            n = G.pic_read_emag_noalloc(ctx.ctx, 0, out)
            assert n == ref.size
            assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
        # after a step the field changes; the fixed scratch must follow
        ctx.step(1)
        ctx.compute_fields()
        ref2 = ctx.fields(G.PIC_FIELD_EMAG)
        out2 = np.empty(ref2.size)
        G.pic_read_emag_noalloc(ctx.ctx, 0, out2)
        assert np.linalg.norm(out2 - ref2) <= 1e-12 * np.linalg.norm(ref2)


def test_noalloc_emag_rejects_meshes_beyond_its_scratch():
    G.build()
    cfg = W.base_config(precision=W.FP32, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, phi_right=1.0)
    with G.Context(cfg) as ctx:
        ctx.set_mesh(0, 512, 512, 1.0 / 512)  # 262,144 leaves > 131,072
        out = np.empty(512 * 512)
        with pytest.raises(G.PicError) as e:
            G.pic_read_emag_noalloc(ctx.ctx, 0, out)
        assert e.value.status == G.PIC_EINVAL and "131072" in str(e.value)
