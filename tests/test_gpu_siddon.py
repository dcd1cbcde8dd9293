"""Siddon system matrix on the GPU against the oracle: the ray-pixel index
pattern and the lengths must match bit for bit (Sec. 2 Eq. 1; both sides
perform the same IEEE double operations, the oracle by sorting all crossings,
the kernel by merging the two monotone crossing sequences)."""
import numpy as np
import pytest

from gpu_util import need_cuda

GEOMS = [(32, 60, 46, 0.0), (17, 23, 29, 0.0), (16, 20, 24, 0.05), (1, 3, 4, 0.0)]


@pytest.mark.gpu
@pytest.mark.parametrize("ns,nv,nb,sl", GEOMS)
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_siddon_dense_and_csr_bit_exact(oracle_mod, ns, nv, nb, sl, storage):
    need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(ns, nv, nb, sqrt_lambda=sl)
    csr = O.siddon_csr(g)
    sysg = ct.System(ct.make_geometry(ns, nv, nb, sl), storage)
    rp, ci, va = sysg.export_csr()
    np.testing.assert_array_equal(rp, csr.row_ptr)
    np.testing.assert_array_equal(ci, csr.col_idx)
    assert va.tobytes() == csr.val.tobytes()
    A = sysg.export_dense()
    Ao = O.dense_system(g, csr)
    if storage == "fp32":
        Ao = Ao.astype(np.float32)
    assert A.tobytes() == np.asfortranarray(Ao).tobytes()


@pytest.mark.gpu
@pytest.mark.parametrize("ns,nv,nb", [(128, 180, 182), (256, 360, 364)])
def test_siddon_csr_bit_exact_full_size(oracle_mod, ns, nv, nb):
    """Full-size geometries of the 128x128 and 256x256 workloads: the whole
    index pattern and every length, against the oracle's CSR."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(ns, nv, nb, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    sysg = ct.System(ct.make_geometry(ns, nv, nb, 0.05), "fp32")
    rp, ci, va = sysg.export_csr()
    np.testing.assert_array_equal(rp, csr.row_ptr)
    np.testing.assert_array_equal(ci, csr.col_idx)
    assert va.tobytes() == csr.val.tobytes()


@pytest.mark.gpu
def test_forward_projection_matches_oracle(oracle_mod):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    from paper_2412_07631_b300 import synth
    O = oracle_mod
    g = O.Geometry(32, 60, 46)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(32, 5, 8)
    P = O.forward(csr, X)
    sysg = ct.System(ct.make_geometry(32, 60, 46), "fp64")
    Pg = sysg.forward(torch.from_numpy(np.ascontiguousarray(X.T)).cuda())
    np.testing.assert_allclose(Pg.cpu().numpy().T, P, rtol=1e-14, atol=1e-12)


# fan beam (the paper's scanner): n_side, sources, detectors, fan_deg, source_dist, sqrt_lambda
FAN = [(16, 24, 21, 30.0, 40.0, 0.0), (24, 36, 33, 25.0, 60.0, 0.05), (32, 48, 64, 33.0, 65.0, 0.0)]


@pytest.mark.gpu
@pytest.mark.parametrize("ns,nv,nd,fan,sid,sl", FAN)
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_fan_beam_siddon_bit_exact(oracle_mod, ns, nv, nd, fan, sid, sl, storage):
    """Fan-beam rays: the host ray tables of both sides are computed with the
    same FP64 operations, so the kernel's index pattern and lengths equal the
    oracle's bit for bit, as in parallel beam."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g = O.Geometry(ns, nv, nd, arc_deg=360.0, sqrt_lambda=sl, kind="fan", source_dist=sid, fan_deg=fan)
    csr = O.siddon_csr(g)
    sysg = ct.System(ct.make_geometry(ns, nv, nd, sl, kind="fan", source_dist=sid, fan_deg=fan), storage)
    rp, ci, va = sysg.export_csr()
    np.testing.assert_array_equal(rp, csr.row_ptr)
    np.testing.assert_array_equal(ci, csr.col_idx)
    assert va.tobytes() == csr.val.tobytes()
    A = sysg.export_dense()
    Ao = O.dense_system(g, csr)
    if storage == "fp32":
        Ao = Ao.astype(np.float32)
    assert A.tobytes() == np.asfortranarray(Ao).tobytes()


@pytest.mark.gpu
def test_fan_beam_geometry_validation():
    need_cuda()
    import paper_2412_07631_b300 as ct
    with pytest.raises(ct.CTQRError):  # source inside the image
        ct.System(ct.make_geometry(32, 10, 20, kind="fan", source_dist=10.0, fan_deg=30.0))
    with pytest.raises(ct.CTQRError):  # fan angle out of range
        ct.System(ct.make_geometry(32, 10, 20, kind="fan", source_dist=60.0, fan_deg=190.0))


@pytest.mark.gpu
@pytest.mark.parametrize("geom", [dict(ns=32, nv=60, nb=46), dict(ns=17, nv=23, nb=29, sl=0.05),
                                  dict(ns=24, nv=36, nb=33, kind="fan", sid=60.0, fan=25.0),
                                  dict(ns=128, nv=180, nb=182, sl=0.05)])
def test_joseph_bit_exact(oracle_mod, geom):
    """Joseph's projector on the GPU against the oracle, parallel and fan
    beam: index pattern and weights bit for bit, dense FP32 copy too."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    ns, nv, nb, sl = geom["ns"], geom["nv"], geom["nb"], geom.get("sl", 0.0)
    if geom.get("kind") == "fan":
        g = O.Geometry(ns, nv, nb, arc_deg=360.0, sqrt_lambda=sl, kind="fan", source_dist=geom["sid"],
                       fan_deg=geom["fan"], projector="joseph")
        cg = ct.make_geometry(ns, nv, nb, sl, kind="fan", source_dist=geom["sid"], fan_deg=geom["fan"],
                              projector="joseph")
    else:
        g = O.Geometry(ns, nv, nb, sqrt_lambda=sl, projector="joseph")
        cg = ct.make_geometry(ns, nv, nb, sl, projector="joseph")
    csr = O.siddon_csr(g)
    sysg = ct.System(cg, "fp32")
    rp, ci, va = sysg.export_csr()
    np.testing.assert_array_equal(rp, csr.row_ptr)
    np.testing.assert_array_equal(ci, csr.col_idx)
    assert va.tobytes() == csr.val.tobytes()
    if ns <= 32:
        A = sysg.export_dense()
        assert A.tobytes() == np.asfortranarray(O.dense_system(g, csr).astype(np.float32)).tobytes()
