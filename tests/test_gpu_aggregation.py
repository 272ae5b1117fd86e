"""GPU parity of the decoupled aggregation (Alg. 4) run on the device: one GPU
thread per tile of consecutive rows, Algorithm 1 on the tile's induced
submatrix.  Aggregate maps are integer work: bit-exact against the oracle's
tiled aggregation, and so are the hierarchies built from them."""

import numpy as np
import pytest

from conftest import oracle_iterate
from oracle import oracle as O
from paper_1209_0960_gb300 import amg
from paper_1209_0960_gb300 import problems as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _oracle_params(prm, **kw):
    d = dict(delta=prm.delta, beta=prm.beta, omega=prm.omega, s_min=prm.s_min,
             s_max=prm.s_max, d_max=prm.d_max, coarsen_target=prm.coarsen_target,
             max_levels=prm.max_levels, dense_cap=prm.dense_cap,
             min_rate=prm.min_coarsen_rate)
    d.update(kw)
    return d


MAPS = {
    "lognormal_tile64": (lambda: P.lognormal3d((20, 18, 16), seed=6), 64),
    "lognormal_tile_ragged": (lambda: P.lognormal3d((20, 18, 16), seed=6), 331),
    "lognormal_tile_4k": (lambda: P.lognormal3d((24, 24, 24), seed=2), 4096),
    "layered_tile_plane": (lambda: P.layered3d((16, 16, 12), seed=1), 256),
    "anisotropic_tile_500": (lambda: P.anisotropic3d((14, 15, 16), seed=2), 500),
    "laplace2d_tile1": (lambda: P.laplace2d_random_rhs(12), 1),
    "laplace2d_tile_gt_n": (lambda: P.laplace2d_random_rhs(20), 1000),
    "hub_graph": (lambda: P.hub_graph2d(40), 97),
    "cube_in_cube": (lambda: P.cube_in_cube3d(16), 200),
}


@pytest.mark.parametrize("case", list(MAPS))
def test_device_tiled_aggregation_matches_oracle(case):
    maker, tile = MAPS[case]
    p = maker()
    prm = amg.amg_params_default(p.dim)
    prm.aggregation_tile = tile
    prm.aggregation_device = 1
    agg1, n1 = amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    agg2, n2 = O.aggregate(p.row_ptr, p.col, p.val, dict(_oracle_params(prm), agg_tile=tile))
    assert n1 == n2 and np.array_equal(agg1, agg2)
    # and the host threads give the same map
    prm.aggregation_device = 0
    agg3, n3 = amg.amg_aggregate(p.row_ptr, p.col, p.val, prm)
    assert n3 == n1 and np.array_equal(agg3, agg1)


@pytest.mark.parametrize("seed", range(2))
def test_device_tiled_aggregation_with_isolated_vertices(seed):
    rng = np.random.default_rng(10 + seed)
    K = np.exp(rng.normal(0.0, 4.0, size=(12, 11, 10)))
    rp, ci, va, b = P.assemble_fv(K, bc=[(1.0, 0.0), (None, None), (None, None)])
    prm = amg.amg_params_default(3)
    prm.beta = 0.02
    prm.aggregation_tile = 150
    prm.aggregation_device = 1
    _, iso, _, _ = O.strength(rp, ci, va, _oracle_params(prm))
    assert iso.sum() > 20
    agg1, n1 = amg.amg_aggregate(rp, ci, va, prm)
    agg2, n2 = O.aggregate(rp, ci, va, dict(_oracle_params(prm), agg_tile=150))
    assert n1 == n2 and np.array_equal(agg1, agg2)


HIER = {
    "lognormal_24_tile512": (lambda: P.lognormal3d((24, 24, 24), seed=3), 512, {"coarsen_target": 200}),
    "layered_20_tile400": (lambda: P.layered3d((20, 20, 20), seed=4), 400, {"coarsen_target": 150}),
}


@pytest.mark.parametrize("case", list(HIER))
def test_device_tiled_hierarchy_matches_oracle(case):
    maker, tile, over = HIER[case]
    p = maker()
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=p.dim, aggregation_tile=tile,
                     aggregation_device=1, **over)
    try:
        H = O.Hierarchy(p.row_ptr, p.col, p.val, _oracle_params(solver.params, agg_tile=tile))
        summary, levels = solver.info()
        assert summary["num_levels"] == H.num_levels >= 3
        for l in range(H.num_levels):
            g, o = solver.level(l), H.level(l)
            assert np.array_equal(g["row_ptr"], o["row_ptr"])
            assert np.array_equal(g["col"], o["col"])
            assert np.array_equal(g["val"].view(np.uint64), o["val"].view(np.uint64)), l
            if l < H.num_levels - 1:
                assert np.array_equal(g["agg"], o["agg"])
                assert np.array_equal(g["colour"], o["colour"])
        # the V-cycle and the solve on the tiled hierarchy
        r = np.random.default_rng(1).standard_normal(p.n)
        z = solver.vcycle(torch.from_numpy(r).cuda())
        torch.cuda.synchronize()
        z_or = H.vcycle(r)
        assert np.abs(z.cpu().numpy() - z_or).max() <= 1e-12 * np.abs(z_or).max()
        x, rc, info = solver.solve(torch.from_numpy(p.b).cuda(), tol=1e-10, maxit=300)
        assert rc == amg.AMG_OK
        xo, it_o, _, _ = H.pcg(p.b, tol=1e-10, maxit=300)
        assert abs(info["iterations"] - it_o) <= 1
        xo = oracle_iterate(H, p.b, info["iterations"], it_o, xo)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
    finally:
        solver.close()


def test_device_and_host_tiles_build_the_same_hierarchy():
    p = P.lognormal3d((32, 32, 32), seed=8)
    a = amg.AMG(p.row_ptr, p.col, p.val, dim=3, aggregation_tile=1024, aggregation_device=1)
    b = amg.AMG(p.row_ptr, p.col, p.val, dim=3, aggregation_tile=1024, aggregation_device=0)
    try:
        sa, _ = a.info()
        sb, _ = b.info()
        assert sa["num_levels"] == sb["num_levels"]
        for l in range(sa["num_levels"] - 1):
            assert np.array_equal(a.level(l)["agg"], b.level(l)["agg"])
    finally:
        a.close()
        b.close()
