"""Multi-instance packs (aim_pack_*): several scatterers through one launch
per product stage.  Each instance's rows of a packed product equal the
instance's own product (complex64 to 1e-5, FP64-accurate to 1e-12) and the
oracle's AIM product of that scatterer; the padding stays zero; a packed solve
gives every instance the solution of its solve alone (both at the solver
tolerance: true residual <= 1e-6, difference within 1e-4)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, random_complex, random_incidence  # noqa: E402
from oracle import aim as oaim  # noqa: E402
from oracle.rwg import RWG  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402

K0 = 2 * np.pi
H = 0.1


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.load()


def sphere(R):
    return icosphere_mesh(R, icosphere_frequency(R))


# closed bodies of different sizes (different grid boxes), one of them CFIE:
# (radius, cfie alpha, right-hand sides)
SPHERES = [(0.3, 1.0, 2), (0.5, 0.6, 3), (0.4, 1.0, 1)]
# planar plates of different sides (planar grids): (side, squares per side, right-hand sides)
PLATES = [(1.0, 9, 2), (1.6, 14, 1), (0.7, 6, 3)]


def _build(items, sphere_kind):
    ctxs, meshes = [], []
    for size, par, nr in items:
        if sphere_kind:
            v, t = sphere(size)
            alpha = par
        else:
            v, t = plate_mesh(size, par)
            alpha = 1.0
        ctxs.append(g.aim_setup(v, t, K0, H, M=2, near_radius=3 * H, max_rhs=nr, precision=g.AIM_C64,
                                cfie_alpha=alpha))
        meshes.append((v, t, alpha))
    return ctxs, meshes


@pytest.fixture(scope="module")
def sphere_pack():
    ctxs, meshes = _build(SPHERES, True)
    pack = g.aim_pack_create(ctxs, [nr for _, _, nr in SPHERES])
    yield pack, ctxs, meshes
    pack.close()
    for c in ctxs:
        c.close()


@pytest.fixture(scope="module")
def plate_pack():
    ctxs, meshes = _build(PLATES, False)
    pack = g.aim_pack_create(ctxs, [nr for _, _, nr in PLATES])
    yield pack, ctxs, meshes
    pack.close()
    for c in ctxs:
        c.close()


def _inputs(pack, seed):
    return [random_complex((nr, c.N), seed=seed + i) for i, (c, nr) in enumerate(zip(pack.ctxs, pack.nrhs))]


def _pick(which, sphere_pack, plate_pack):
    return sphere_pack if which == "sphere" else plate_pack


@pytest.mark.parametrize("which", ["sphere", "plate"])
def test_packed_product_equals_each_instance_alone(which, sphere_pack, plate_pack):
    pack, ctxs, _ = _pick(which, sphere_pack, plate_pack)
    xs = _inputs(pack, 3)
    x128 = pack.pack([torch.from_numpy(x).cuda() for x in xs])
    assert x128.shape == (pack.B, pack.ld)
    # complex64: one launch per stage for all instances
    y64 = g.aim_pack_matvec(pack, x128.to(torch.complex64).contiguous(), precision=g.AIM_C64)
    y128 = g.aim_pack_matvec(pack, x128, precision=g.AIM_C128)
    torch.cuda.synchronize()
    for i, (ctx, x) in enumerate(zip(ctxs, xs)):
        r0, r1, n = pack.rows(i)
        alone64 = g.aim_matvec(ctx, torch.from_numpy(x).to(torch.complex64).cuda(), precision=g.AIM_C64)
        alone128 = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=g.AIM_C128)
        torch.cuda.synchronize()
        a64, a128 = alone64.cpu().numpy(), alone128.cpu().numpy()
        assert rel(y64[r0:r1, :n].cpu().numpy(), a128) <= 1e-5, i
        assert rel(a64, a128) <= 1e-5
        assert rel(y128[r0:r1, :n].cpu().numpy(), a128) <= 1e-12, i
        # the padding of the instance's rows is zero
        assert torch.count_nonzero(y64[r0:r1, n:]).item() == 0
        assert torch.count_nonzero(y128[r0:r1, n:]).item() == 0


@pytest.mark.parametrize("which", ["sphere", "plate"])
def test_packed_product_matches_oracle(which, sphere_pack, plate_pack):
    pack, _, meshes = _pick(which, sphere_pack, plate_pack)
    xs = _inputs(pack, 11)
    x = pack.pack([torch.from_numpy(v).cuda() for v in xs])
    y64 = g.aim_pack_matvec(pack, x.to(torch.complex64).contiguous(), precision=g.AIM_C64).cpu().numpy()
    y128 = g.aim_pack_matvec(pack, x, precision=g.AIM_C128).cpu().numpy()
    for i, ((v, t, alpha), xi) in enumerate(zip(meshes, xs)):
        op = oaim.AIMOperator(RWG(v, t), K0, H, 2, near_radius=3 * H, alpha=alpha)
        ref = op.matvec(xi)
        r0, r1, n = pack.rows(i)
        assert rel(y64[r0:r1, :n], ref) <= 1e-5, i
        assert rel(y128[r0:r1, :n], ref) <= 1e-12, i


def test_packed_solve_matches_solves_alone(sphere_pack):
    pack, ctxs, _ = sphere_pack
    rng = np.random.default_rng(4)
    Vs = []
    for ctx, nr in zip(ctxs, pack.nrhs):
        kh, po = random_incidence((nr + 1) // 2, rng=rng)
        Vs.append(g.aim_rhs_planewave(ctx, kh[:nr], po[:nr]))
    V = pack.pack(Vs)
    X, info = g.aim_pack_solve(pack, V, tol=1e-6)
    assert info["converged"].all() and info["rel_res"].max() <= 1e-6
    assert torch.count_nonzero(pack.pack(pack.unpack(X)) - X).item() == 0  # the padding stays zero
    for i, ctx in enumerate(ctxs):
        Xi = pack.unpack(X)[i].contiguous()
        alone, inf = g.aim_solve(ctx, Vs[i].clone(), tol=1e-6)
        assert inf["converged"].all()
        a = alone.cpu().numpy()
        assert np.linalg.norm(Xi.cpu().numpy() - a) <= 1e-4 * np.linalg.norm(a), i
        # true residual of the packed solution with the instance's own FP64-accurate product
        r = torch.linalg.norm(Vs[i] - g.aim_matvec(ctx, Xi, precision=g.AIM_C128), dim=1) / torch.linalg.norm(
            Vs[i], dim=1)
        assert r.max().item() <= 1.01e-6, i


def test_pack_rejects_mismatched_contexts():
    v, t = plate_mesh(1.0, 9)
    a = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64)
    b = g.aim_setup(v, t, K0, 0.12, max_rhs=2, precision=g.AIM_C64)  # another grid step
    s = g.aim_setup(*sphere(0.3), K0, H, max_rhs=1, precision=g.AIM_C64)  # a three-dimensional grid
    try:
        for ctxs, nr in (([a, b], [1, 1]), ([a, s], [1, 1]), ([a], [3]), ([a, a], [1, 1]), ([a], [0])):
            with pytest.raises(g.AIMError) as e:
                g.aim_pack_create(ctxs, nr)
            assert e.value.code == 1  # AIM_EINVAL
        p = g.aim_pack_create([a], [2])  # one instance is a pack too
        x = torch.zeros((p.B, p.ld), dtype=torch.complex64, device="cuda")
        with pytest.raises(g.AIMError):
            g.aim_pack_matvec(p, x, x, precision=g.AIM_C64)  # x and y overlap
        p.close()
    finally:
        for c in (a, b, s):
            c.close()


def test_packed_tfqmr_solve_matches_gmres():
    """A pack takes its Krylov method from its first context: TFQMR on two
    plates gives every instance the GMRES solution to the tolerance."""
    ctxs = []
    for side, n in ((1.0, 9), (1.3, 12)):
        v, t = plate_mesh(side, n)
        ctxs.append(g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64, krylov=g.AIM_TFQMR))
    try:
        kh, po = random_incidence(1, seed=6)
        Vs = [g.aim_rhs_planewave(c, kh, po) for c in ctxs]
        pack = g.aim_pack_create(ctxs, [2, 2])
        X, info = g.aim_pack_solve(pack, pack.pack(Vs), tol=1e-6)
        assert info["converged"].all() and info["rel_res"].max() <= 1e-6
        for i, c in enumerate(ctxs):
            g.aim_set_krylov(c, g.AIM_GMRES)
            Xg, _ = g.aim_solve(c, Vs[i].clone(), tol=1e-6)
            a = Xg.cpu().numpy()
            assert np.linalg.norm(pack.unpack(X)[i].cpu().numpy() - a) <= 1e-4 * np.linalg.norm(a)
        pack.close()
    finally:
        for c in ctxs:
            c.close()
