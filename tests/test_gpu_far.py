"""nf_derivatives / nf_far_forces against the FP64 far-field oracle
(Sec. "Far-field Computation"), and near + far against plain Ewald sums."""
import numpy as np
import pytest

import oracle

from _helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[0, 1], ids=["fp64", "double-float"])
def arith(request):
    """Runs a test with each arithmetic of the per-particle far-field kernels."""
    from paper_2110_11392_gb300 import _lib
    before = _lib.nf_far_get_arith()
    _lib.nf_far_set_arith(request.param)
    yield request.param
    _lib.nf_far_set_arith(before)


def _uniform(N, seed):
    pos = np.random.default_rng(seed).random((N, 3)).astype(np.float32)
    pos[pos >= 1.0] = 0.0
    return pos


def _clustered(N, K, seed):
    from workloads import config_plain
    return config_plain(N=N, K=K, seed=seed).pos


def _dr_gpu(ff):
    """The compressed transformed derivatives of a derivatives buffer,
    [nt][K][K][K/2+1] reals: real parts of even terms, imaginary parts of odd ones."""
    head = ff.derivs[:256].cpu().numpy()
    o_dh = int(np.frombuffer(head[72:80].tobytes(), np.uint64)[0])   # DerivHeader.o_dh
    K, nt = ff.K, ff.nterms
    n = nt * K * K * (K // 2 + 1)
    raw = ff.derivs[o_dh:o_dh + 8 * n].cpu().numpy()
    return np.frombuffer(raw.tobytes(), np.float64).reshape(nt, K, K, K // 2 + 1)


@pytest.mark.parametrize("K,R,p,box", [(5, 2, 4, 1.0), (8, 2, 8, 1.0), (11, 2, 8, 1.0), (9, 3, 6, 3.0),
                                       (6, 2, 12, 1.0), (4, 1, 6, 1.0)])
def test_derivatives_match_oracle(K, R, p, box):
    import paper_2110_11392_gb300 as nf
    ff = nf.FarField(K, R, p, box)
    D = oracle.derivatives(K, R, p, box)          # another Ewald split than the library's
    ref = np.fft.rfftn(D.reshape(K, K, K, -1), axes=(0, 1, 2)).transpose(3, 0, 1, 2)
    order = np.array([sum(t) for t in oracle.multipole_index(p)])
    odd = (order % 2 == 1)[:, None, None, None]
    # rounding is relative to the size of the derivatives of the same order: a term
    # that vanishes by the grid's symmetry (e.g. (3,1,1) on K = 4) has only noise as
    # its own scale, so every term is measured against the largest of its order
    per_term = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)
    per_order = {o: per_term[order == o].max() for o in set(order)}
    scale = np.array([per_order[o] for o in order])[:, None, None, None]
    # the parity the library relies on: even terms transform to reals, odd to imaginaries
    dropped = np.where(odd, ref.real, ref.imag)
    assert (np.abs(dropped) / scale).max() < 1e-12
    kept = np.where(odd, ref.imag, ref.real)
    got = _dr_gpu(ff)
    assert (np.abs(got - kept) / scale).max() < 1e-10


@pytest.mark.parametrize("K,R,p", [(8, 2, 8), (5, 2, 4), (16, 3, 6)])
def test_double_float_copy_of_derivatives(K, R, p):
    """The buffer also holds the transformed derivatives as double-float pairs
    (for the double-float k-space product, any K): hi = fp32(D), lo = fp32(D - hi)."""
    import paper_2110_11392_gb300 as nf
    ff = nf.FarField(K, R, p)
    head = ff.derivs[:256].cpu().numpy()
    o_drdf = int(np.frombuffer(head[136:144].tobytes(), np.uint64)[0])   # DerivHeader.o_drdf
    assert o_drdf != 0
    D = _dr_gpu(ff).ravel()
    pairs = ff.derivs[o_drdf:o_drdf + 8 * D.size].cpu().numpy().view(np.float32).reshape(-1, 2)
    hi = D.astype(np.float32)
    assert np.array_equal(pairs[:, 0], hi)
    assert np.array_equal(pairs[:, 1], (D - hi.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("K,R,p,N,kind", [(5, 2, 4, 3000, "uniform"), (8, 2, 8, 20000, "clustered"),
                                          (11, 2, 8, 65536, "uniform"), (7, 3, 5, 9000, "clustered"),
                                          (16, 2, 8, 40000, "clustered"), (6, 2, 1, 500, "uniform"),
                                          (6, 1, 7, 8000, "clustered"), (4, 1, 6, 2000, "uniform"),
                                          (13, 2, 4, 4000, "uniform"), (10, 2, 6, 6000, "clustered")])
def test_far_forces_match_oracle(K, R, p, N, kind, arith):
    import torch
    import paper_2110_11392_gb300 as nf
    pos = _uniform(N, 21) if kind == "uniform" else _clustered(N, K, 22)
    ff = nf.FarField(K, R, p)
    a, T = ff(to_dev(pos), want_taylors=True)
    torch.cuda.synchronize()
    aref, Tref = oracle.far_field(pos, 1.0, K, R, p, return_taylors=True)
    T = T.cpu().numpy()
    tscale = np.abs(Tref).max(axis=0) + 1e-300
    assert (np.abs(T - Tref).max(axis=0) / tscale).max() < 1e-10
    a = a.cpu().numpy()
    assert np.abs(a - aref).max() < 1e-10 * np.abs(aref).max()
    rel = np.linalg.norm(a - aref, axis=1) / np.linalg.norm(aref, axis=1)
    assert np.median(rel) < 1e-11


def test_add_to_near_field_output():
    import torch
    import paper_2110_11392_gb300 as nf
    pos = to_dev(_uniform(8000, 5))
    ff = nf.FarField(8, 2, 6)
    near = nf.forces(pos, 1.0, 8, 2, 1e-4)
    far = ff(pos)
    tot = near.clone()
    ff(pos, add_to=tot, want_far=False)
    torch.cuda.synchronize()
    assert torch.equal(tot, near + far.float())


def test_total_force_matches_ewald_at_the_papers_configuration():
    # 65536 random particles, CPD 11, order 8 (Sec. "Ewald"); FP32 near field
    # plus FP64 far field against plain Ewald sums.
    import torch
    import paper_2110_11392_gb300 as nf
    N, K, R, p = 65536, 11, 2, 8
    pos = _uniform(N, 11)
    eps = 1e-5
    d = to_dev(pos)
    tot = nf.forces(d, 1.0, K, R, eps)
    nf.FarField(K, R, p)(d, add_to=tot, want_far=False)
    torch.cuda.synchronize()
    sinks = np.sort(np.random.default_rng(11).choice(N, 256, replace=False))
    ref = oracle.ewald_forces(pos, 1.0, sinks=sinks)
    fe = oracle.frac_error(tot.cpu().numpy()[sinks].astype(np.float64), ref)
    assert np.median(fe) < 2.4e-5 and np.percentile(fe, 99) < 3.2e-4


def test_single_particle_and_lattice():
    import torch
    import paper_2110_11392_gb300 as nf
    ff = nf.FarField(8, 2, 8)
    one = ff(to_dev(np.array([[0.37, 0.61, 0.12]], np.float32)))
    g = (np.arange(8) + 0.5) / 8
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    a = ff(to_dev(lat))
    torch.cuda.synchronize()
    assert one.abs().max().item() < 1e-12
    assert a.abs().max().item() < 1e-12 * (1.0 / 512) * 64


def test_graph_replay_is_bit_identical():
    import torch
    import paper_2110_11392_gb300 as nf
    pos = to_dev(_clustered(30000, 10, 4))
    ff = nf.FarField(10, 2, 8)
    ws = ff.workspace(30000)
    eager = ff(pos, ws=ws)
    out = torch.zeros_like(eager)
    from paper_2110_11392_gb300 import _lib
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    # one call on the capture stream first (kernel attributes are set outside the capture)
    _lib.nf_far_forces(pos, 1.0, ff.K, ff.R, ff.p, ff.derivs, out, None, None, ws, stream=s)
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        _lib.nf_far_forces(pos, 1.0, ff.K, ff.R, ff.p, ff.derivs, out, None, None, ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_argument_errors():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    ff = nf.FarField(8, 2, 4)
    pos = to_dev(_uniform(100, 1))
    ws = ff.workspace(100)
    acc = torch.empty((100, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.NFError):   # derivatives made for another R
        _lib.nf_far_forces(pos, 1.0, 8, 3, 4, ff.derivs, acc, None, None, ws)
    with pytest.raises(_lib.NFError):   # another box side
        _lib.nf_far_forces(pos, 2.0, 8, 2, 4, ff.derivs, acc, None, None, ws)
    with pytest.raises(_lib.NFError):   # too small a buffer for K = 9
        _lib.nf_far_forces(pos, 1.0, 9, 2, 4, ff.derivs, acc, None, None, ws)
    with pytest.raises(_lib.NFError):   # workspace too small
        _lib.nf_far_forces(pos, 1.0, 8, 2, 4, ff.derivs, acc, None, None, ws[:1024])
    assert _lib.nf_derivatives_bytes(8, 13) == 0
    with pytest.raises(_lib.NFError):
        nf.FarField(4, 2, 4)            # K < 2R + 1 is caught by the library


@pytest.mark.parametrize("K,p", [(6, 12), (5, 10), (8, 12)])
def test_highest_orders_match_oracle(K, p, arith):
    import torch
    import paper_2110_11392_gb300 as nf
    pos = _uniform(2000, 31)
    a = nf.FarField(K, 2, p)(to_dev(pos))
    torch.cuda.synchronize()
    aref = oracle.far_field(pos, 1.0, K, 2, p)
    assert np.abs(a.cpu().numpy() - aref).max() < 1e-10 * np.abs(aref).max()


def test_sparse_cells_faces_and_wrapping(arith):
    # far fewer particles than cells (most cells empty), particles on cell
    # faces, and coordinates outside [0, box) that must wrap like nf_forces
    import torch
    import paper_2110_11392_gb300 as nf
    K = 12
    rng = np.random.default_rng(8)
    pos = rng.random((300, 3))
    pos[:40] = np.round(pos[:40] * K) / K                    # exactly on faces
    pos[40:80] += rng.integers(-3, 4, size=(40, 3))          # whole boxes away
    pos = pos.astype(np.float32)
    a = nf.FarField(K, 2, 6)(to_dev(pos))
    torch.cuda.synchronize()
    aref = oracle.far_field(pos, 1.0, K, 2, 6)
    assert np.abs(a.cpu().numpy() - aref).max() < 1e-10 * np.abs(aref).max()
    # the same particles moved by whole boxes feel the same force
    b = nf.FarField(K, 2, 6)(to_dev(((pos.astype(np.float64) % 1.0) % 1.0).astype(np.float32)))
    torch.cuda.synchronize()
    assert np.abs(a.cpu().numpy() - b.cpu().numpy()).max() < 1e-6 * np.abs(aref).max()


def test_release_changes_nothing():
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    pos = to_dev(_uniform(3000, 2))
    ff = nf.FarField(7, 2, 5)
    a = ff(pos)
    _lib.nf_far_release()
    b = ff(pos)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_total_force_call_equals_near_plus_far():
    import torch
    import paper_2110_11392_gb300 as nf
    pos = to_dev(_clustered(20000, 9, 12))
    ff = nf.FarField(9, 2, 6)
    eps = 1e-3
    near = nf.forces(pos, 1.0, 9, 2, eps)
    ref = near.clone()
    ff(pos, add_to=ref, want_far=False)
    tot = ff.total(pos, eps)
    torch.cuda.synchronize()
    assert torch.equal(tot, ref)


@pytest.mark.parametrize("K", [11, 12, 16, 24, 32, 64, 96, 128])
def test_the_two_arithmetics_agree(K):
    """The FP64 mode runs the mixed-radix transforms in FP64 and the FP64
    product for every K; the double-float mode the mixed-radix transforms in
    double-float for K = 11 (prime), 12, 24 and 96 (factors 4, 2, 3) and the
    radix-4/2 ones for K = 16, 32, 64, 128 (powers of two), with the
    double-float product.  K = 64 splits each line pass of the radix-4/2
    kernels into two blocks per row (33 frequencies, 32 per block) and the z
    pass into three field chunks; K = 128 (the grid of the 512^3 box) into
    five and six."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    pos = to_dev(_clustered(60000, K, 13))
    ff = nf.FarField(K, 2, 8)
    before = _lib.nf_far_get_arith()
    try:
        _lib.nf_far_set_arith(_lib.NF_FAR_FP64)
        a64, t64 = ff(pos, want_taylors=True)
        _lib.nf_far_set_arith(_lib.NF_FAR_DOUBLE_FLOAT)
        adf, tdf = ff(pos, want_taylors=True)
        adf_only = ff(pos)  # forces alone: the Taylors are rebuilt in double-float only
        torch.cuda.synchronize()
    finally:
        _lib.nf_far_set_arith(before)
    scale = a64.abs().max().item()
    assert (a64 - adf).abs().max().item() < 1e-12 * scale
    # the double-float forces do not depend on whether the FP64 Taylors are asked for
    assert torch.equal(adf_only, adf)
    tscale = t64.abs().amax(dim=0) + 1e-300
    assert ((t64 - tdf).abs().amax(dim=0) / tscale).max().item() < 1e-12
    with pytest.raises(_lib.NFError):
        _lib.nf_far_set_arith(2)


def test_largest_power_of_two_grid_in_both_arithmetics():
    """K = 256, the largest grid of the radix-4/2 double-float transforms (8 fields per line
    block, 16 per z block): the double-float far field equals the FP64 one (mixed-radix
    transforms) to 1e-12.  Low order and few particles keep the buffers small."""
    import torch
    import paper_2110_11392_gb300 as nf
    from paper_2110_11392_gb300 import _lib
    K = 256
    pos = to_dev(_uniform(30000, 17))
    ff = nf.FarField(K, 2, 2)
    before = _lib.nf_far_get_arith()
    try:
        _lib.nf_far_set_arith(_lib.NF_FAR_FP64)
        a64 = ff(pos)
        _lib.nf_far_set_arith(_lib.NF_FAR_DOUBLE_FLOAT)
        adf = ff(pos)
        torch.cuda.synchronize()
    finally:
        _lib.nf_far_set_arith(before)
    scale = a64.abs().max().item()
    assert scale > 0
    assert (a64 - adf).abs().max().item() < 1e-12 * scale
