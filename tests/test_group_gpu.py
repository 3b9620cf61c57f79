"""Several frequencies solved as one group (hz_solve_group), each context on
its own CUDA stream, against the oracle and against the same contexts solved
one at a time.  Workload: a 192 x 192 smooth random medium with uneven layers
and cells (24-64 points) at 6, 8 and 10 points per wavelength."""
import numpy as np
import pytest

import hz_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-8)])
def test_group_matches_oracle_and_single(precision, tol):
    probs = I.uneven_multifreq(n=192, n_pml=10, seed=4, part_seed=40)
    prec = hz.HZ_MIXED if precision == "mixed" else hz.HZ_FP64
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs, fs, refs = [], [], []
    for pb, s in zip(probs, streams):
        C_pml = O.default_pml_C(pb.m)
        f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, 5)
        box = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml)
        refs.append(box.factor().solve(f))
        c = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=prec, pml_C=C_pml,
                       layer_rows=pb.layer_rows, cell_cols=pb.cell_cols, stream=s.cuda_stream)
        c.hz_factor()
        ctxs.append(c)
        fs.append(f)
    us, sts = hz.hz_solve_group(ctxs, fs)
    singles = [c.hz_solve(f)[0] for c, f in zip(ctxs, fs)]
    for c in ctxs:
        c.close()
    for u, s1, ref, st in zip(us, singles, refs, sts):
        assert _rel(u, ref) < tol
        assert st.resid < 1e-8
        assert st.iterations > 0
        # the group runs each member's kernels in the same order as a lone solve
        assert _rel(u, s1) < 1e-12


def test_group_device_pointers_and_errors():
    pb = I.smooth_random(64, n_pml=8, L=3, C=3, seed=81, ppw=8, corr_pts=8)
    C_pml = O.default_pml_C(pb.m)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 2, 82)
    ref = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml).factor().solve(f)
    a = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_FP64, pml_C=C_pml,
                   device_ptrs=True)
    b = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED, pml_C=C_pml,
                   device_ptrs=True)
    a.hz_factor()
    fd = torch.from_numpy(f).cuda()
    # a context listed twice, a member not factored, precisions that differ
    with pytest.raises(hz.HzError):
        hz.hz_solve_group([a, a], [fd, fd])
    with pytest.raises(hz.HzError):
        hz.hz_solve_group([a, b], [fd, fd])
    b.hz_factor()
    with pytest.raises(hz.HzError):
        hz.hz_solve_group([a, b], [fd, fd])
    (u,), (st,) = hz.hz_solve_group([a], [fd])
    torch.cuda.synchronize()
    assert _rel(u.cpu().numpy(), ref) < 1e-8
    a.close()
    b.close()


def test_autotuned_sweeps_match_oracle_and_fill_cache(tmp_path, monkeypatch):
    # the tuner times the sweep launch configurations at first use and records
    # its choice per launch shape in the JSON cache
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("HZ_TUNE_CACHE", str(cache))
    pb = I.smooth_random(96, n_pml=8, L=3, C=4, seed=91, ppw=8, corr_pts=8)
    C_pml = O.default_pml_C(pb.m)
    f = I.random_sources(pb.shape_ext, pb.n_pml, 20, 92)
    ref = O.Box(pb.m, pb.n_x, pb.n_z, pb.n_pml, pb.omega, pb.h, C_pml).factor().solve(f)
    # dense inner factors: the tuner chooses the launch shape of the dense block-LU sweep
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=hz.HZ_MIXED,
                     pml_C=C_pml, autotune=True, compress=0.0)
    ctx.hz_factor()
    u, st = ctx.hz_solve(f)
    u2, _ = ctx.hz_solve(f)
    ctx.close()
    assert _rel(u, ref) < 1e-5 and _rel(u2, ref) < 1e-5
    assert st.resid < 1e-8
    import json
    table = json.loads(cache.read_text())
    assert any(k.startswith("sweep es=8") for k in table)
    assert all(isinstance(v, int) and v >= 0 for v in table.values())  # a candidate index per shape
