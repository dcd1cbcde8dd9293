"""Disk tier of the out-of-core path (the matrix in a file of column blocks,
a pinned block cache, background I/O): the disk build equals the in-core
build bit for bit; the disk factorisation equals the host-memory one bit for
bit under the same budget and solves like the in-core one against the FP64
oracle; an interrupted factorisation resumes to the same bits (in the same
process, after reopening the file, and after a write-back that was left half
done); a factored file reopens without recomputation."""
import struct

import numpy as np
import pytest

from gpu_util import need_cuda, rel_err_cols
from paper_2412_07631_b300 import synth

NS, NV, NBINS, SL = 24, 40, 36, 0.05
NB = 64  # file block = outer block: 9 blocks of 64 columns (n = 576)


def _case(O, k=3):
    g = O.Geometry(NS, NV, NBINS, sqrt_lambda=SL)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(NS, k, 8, 4321)
    B = synth.poisson_sinogram(O.forward(csr, X), NS, 1e4, seed=4321)
    return g, csr, B


def _budget(rows, lda, es, nb_outer, width):
    """Device bytes for two staging buffers of one outer block plus `width` columns."""
    stage = es * (-(-rows // 32) * 32) * nb_outer
    return 2 * stage + es * lda * width


def _geom(ct):
    return ct.make_geometry(NS, NV, NBINS, SL)


def _disk(ct, tmp_path, name, storage="fp32", cache=1 << 30, block_cols=NB):
    return ct.System(_geom(ct), storage, disk_path=str(tmp_path / name), host_cache=cache,
                     block_cols=block_cols)


@pytest.mark.gpu
@pytest.mark.parametrize("storage,bc", [("fp32", 64), ("fp64", 32), ("fp32", 96)])
def test_disk_build_equals_device_build(tmp_path, storage, bc):
    need_cuda()
    import paper_2412_07631_b300 as ct
    dev = ct.System(_geom(ct), storage)
    disk = _disk(ct, tmp_path, "a.ctqrd", storage, block_cols=bc)
    assert disk.disk_progress() == (0, 0)
    np.testing.assert_array_equal(dev.export_dense(), disk.export_dense())
    rp0, ci0, va0 = dev.export_csr()
    rp1, ci1, va1 = disk.export_csr()
    np.testing.assert_array_equal(rp0, rp1)
    np.testing.assert_array_equal(va0, va1)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32", "fp64"])
def test_disk_factor_equals_host_tier(tmp_path, precision):
    """Same superpanels, same kernels: the file tier's factors and solves are
    the host tier's, bit for bit."""
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    storage = "fp64" if precision == "fp64" else "fp32"
    es = 8 if storage == "fp64" else 4
    disk = _disk(ct, tmp_path, "f.ctqrd", storage)
    budget = _budget(disk.rows, disk.lda, es, NB, 128)  # superpanels of 128 columns: 5
    host = ct.System(_geom(ct), storage, host_budget=budget)
    Fh = host.factor_ooc(precision, device_budget=budget, nb_outer=NB)
    ct.disk_stats(reset=True)
    Fd = disk.factor_ooc(precision, device_budget=budget, nb_outer=NB)
    io = ct.disk_stats()
    VRh, tauh = Fh.export()
    VRd, taud = Fd.export()
    np.testing.assert_array_equal(VRh, VRd)
    np.testing.assert_array_equal(tauh, taud)
    assert io["bytes_written"] > 0 and io["hits"] > 0  # the cache holds every block here
    dt = torch.float64
    B = torch.rand(4, disk.m, dtype=dt, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    xh = Fh.solve(B, max_iter=3, allow_noconv=True)
    xd = Fd.solve(B, max_iter=3, allow_noconv=True)
    assert torch.equal(xh, xd)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("tf32", 1e-6),
                                           ("bf16", 1e-6)])
def test_disk_factor_matches_oracle(oracle_mod, tmp_path, precision, tol):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    O = oracle_mod
    g, csr, B = _case(O)
    Xo, _, _ = O.qr_solve(g, O.dense_system(g, csr), B)
    storage = "fp64" if precision == "fp64" else "fp32"
    es = 8 if storage == "fp64" else 4
    disk = _disk(ct, tmp_path, "o.ctqrd", storage, cache=0)  # three cache slots
    budget = _budget(disk.rows, disk.lda, es, NB, 192)
    F = disk.factor_ooc(precision, device_budget=budget, nb_outer=NB)
    dt = torch.float32 if precision == "fp32" else torch.float64
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).to(dt).cuda()
    Xg = F.solve(Bt, max_iter=20, tol=1e-10, allow_noconv=True).double().cpu().numpy().T
    err = rel_err_cols(Xg, Xo)
    print(precision, "disk max rel err", err.max(), F.last_info)
    assert err.max() <= tol


def _reference(ct, tmp_path, budget, precision="tf32"):
    ref = _disk(ct, tmp_path, "ref.ctqrd")
    F = ref.factor_ooc(precision, device_budget=budget, nb_outer=NB)
    return F.export()


@pytest.mark.gpu
def test_disk_resume_in_process_is_bit_exact(tmp_path):
    need_cuda()
    import paper_2412_07631_b300 as ct
    disk = _disk(ct, tmp_path, "r.ctqrd")
    budget = _budget(disk.rows, disk.lda, 4, NB, 128)
    VR0, tau0 = _reference(ct, tmp_path, budget)
    assert disk.factor_ooc("tf32", device_budget=budget, stop_after=1) is None
    assert disk.disk_progress() == (1, 128)
    assert disk.factor_ooc("tf32", device_budget=budget, stop_after=2) is None
    assert disk.disk_progress() == (1, 384)
    with pytest.raises(ct.CTQRError):  # another precision cannot continue this file
        disk.factor_ooc("bf16", device_budget=budget)
    F = disk.factor_ooc("tf32", device_budget=budget)
    VR1, tau1 = F.export()
    np.testing.assert_array_equal(VR0, VR1)
    np.testing.assert_array_equal(tau0, tau1)


@pytest.mark.gpu
def test_disk_resume_after_reopen_is_bit_exact(tmp_path):
    need_cuda()
    import paper_2412_07631_b300 as ct
    path = str(tmp_path / "o.ctqrd")
    disk = ct.System(_geom(ct), "fp32", disk_path=path, block_cols=NB)
    budget = _budget(disk.rows, disk.lda, 4, NB, 128)
    VR0, tau0 = _reference(ct, tmp_path, budget)
    assert disk.factor_ooc("tf32", device_budget=budget, stop_after=2) is None
    disk.free()  # as if the process had ended
    again = ct.System.open_disk(path, host_cache=1 << 28)
    assert again.disk_progress() == (1, 256)
    with pytest.raises(ct.CTQRError):  # the file no longer holds A~
        again.export_dense()
    F = again.factor_ooc("tf32", device_budget=budget)
    VR1, tau1 = F.export()
    np.testing.assert_array_equal(VR0, VR1)
    np.testing.assert_array_equal(tau0, tau1)


def _fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for c in b:
        h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


# byte offsets in the file header: magic 8, version 4, element size 4,
# geometry 80, m n rows lda (8 each), bw nblocks state prec nb_inner pad
# (4 each), done_cols, dirty_cols, rjj_min, rjj_max (8 each), checksum
_DONE, _DIRTY, _SUM = 16 + 80 + 32 + 24, 16 + 80 + 32 + 24 + 8, 16 + 80 + 32 + 24 + 32


@pytest.mark.gpu
def test_disk_half_written_superpanel_is_rebuilt(tmp_path):
    """A run that died during a write-back leaves [done, dirty) partly
    rewritten: the resume rebuilds those columns from the sparse rows and
    reaches the same factors."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    path = tmp_path / "h.ctqrd"
    disk = ct.System(_geom(ct), "fp32", disk_path=str(path), block_cols=NB)
    budget = _budget(disk.rows, disk.lda, 4, NB, 128)
    VR0, tau0 = _reference(ct, tmp_path, budget)
    assert disk.factor_ooc("tf32", device_budget=budget, stop_after=1) is None
    disk.free()
    raw = bytearray(path.read_bytes())
    done, dirty = struct.unpack_from("<qq", raw, _DONE)
    assert (done, dirty) == (128, 128)
    # garbage over the first block of the next superpanel, recorded as dirty
    b2 = 4096
    rows_of = lambda b: min(disk.rows, disk.m + min(disk.n, (b + 1) * NB))  # noqa: E731
    for b in range(2):
        b2 += -(-4 * rows_of(b) * NB // 4096) * 4096
    raw[b2:b2 + 4096 * 8] = bytes(range(256)) * 128
    struct.pack_into("<q", raw, _DIRTY, 256)
    struct.pack_into("<Q", raw, _SUM, _fnv1a(bytes(raw[:_SUM])))
    path.write_bytes(bytes(raw))
    again = ct.System.open_disk(str(path))
    F = again.factor_ooc("tf32", device_budget=budget)
    VR1, tau1 = F.export()
    np.testing.assert_array_equal(VR0, VR1)
    np.testing.assert_array_equal(tau0, tau1)


@pytest.mark.gpu
def test_disk_factored_file_reopens_without_recomputation(tmp_path):
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    path = str(tmp_path / "d.ctqrd")
    disk = ct.System(_geom(ct), "fp32", disk_path=path, block_cols=NB)
    budget = _budget(disk.rows, disk.lda, 4, NB, 192)
    F = disk.factor_ooc("tf32", device_budget=budget)
    B = torch.rand(3, disk.m, dtype=torch.float64, device="cuda",
                   generator=torch.Generator("cuda").manual_seed(9))
    x1 = F.solve(B, max_iter=5, allow_noconv=True).clone()
    VR1, _ = F.export()
    F.free()  # closes the file, which stays on disk
    disk.free()
    again = ct.System.open_disk(path)
    assert again.disk_progress() == (2, NS * NS)
    ct.disk_stats(reset=True)
    G = again.factor_ooc("tf32", device_budget=budget)
    io = ct.disk_stats()
    assert io["bytes_written"] <= 8192  # the header only: nothing was factored again
    VR2, _ = G.export()
    np.testing.assert_array_equal(VR1, VR2)
    x2 = G.solve(B, max_iter=5, allow_noconv=True)
    assert torch.equal(x1, x2)
    with pytest.raises(ct.CTQRError):  # the file is the checkpoint
        G.save(str(tmp_path / "x.ctqr"))


@pytest.mark.gpu
def test_disk_small_cache_same_bits(tmp_path):
    """Three cache slots (every V block read back from the file) or a cache
    that holds the whole matrix: the same factors."""
    need_cuda()
    import paper_2412_07631_b300 as ct
    small = _disk(ct, tmp_path, "s.ctqrd", cache=0)
    budget = _budget(small.rows, small.lda, 4, NB, 128)
    ct.disk_stats(reset=True)
    Fs = small.factor_ooc("tf32", device_budget=budget)
    io_small = ct.disk_stats(reset=True)
    VRs, taus = Fs.export()
    VR0, tau0 = _reference(ct, tmp_path, budget)
    io_big = ct.disk_stats()
    np.testing.assert_array_equal(VR0, VRs)
    np.testing.assert_array_equal(tau0, taus)
    assert io_small["misses"] + io_small["prefetched"] > 0
    # with the small cache, the earlier V blocks come back from the file
    assert io_small["bytes_read"] > io_big["bytes_read"]
