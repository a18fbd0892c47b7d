"""C-ABI behaviour on the GPU: error reporting, host end-to-end, batches, profiling, tuner."""
import numpy as np
import pytest

from gpu_helpers import gpu_solve, oracle_solve, phi_rel_err
from paper_2602_02507_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_nonfinite_density_is_reported(prec):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=8, n_theta=16, n_phi=32, L=4)
    m = w.mesh
    rho = torch.from_numpy(w.rho).cuda()
    rho.view(-1)[1234] = float("nan")
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        mesh.set_density(rho)
        mesh.solve()
        with pytest.raises(mpl.MultipoleError) as ei:
            mesh.synchronize()
        assert ei.value.name == "MP_ERR_NONFINITE"
        mesh.synchronize()  # the error word was cleared


@pytest.mark.parametrize("value", [float("inf"), 1e39])
def test_density_beyond_float32_is_reported_on_the_split_path(value):
    """The split path converts the density to float32: a magnitude of 2^128 or more (or an
    infinity) cannot be represented and is reported, whichever conversion path the chunk
    takes (a zero in the same chunk sends it through the checked conversion)."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=8, n_theta=16, n_phi=32, L=4)
    m = w.mesh
    for with_zero in (False, True):
        rho = torch.from_numpy(w.rho).cuda()
        rho.view(-1)[1234] = value
        if with_zero:
            rho.view(-1)[1235] = 0.0
        with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh:
            mesh.set_density(rho)
            mesh.solve()
            with pytest.raises(mpl.MultipoleError) as ei:
                mesh.synchronize()
            assert ei.value.name == "MP_ERR_NONFINITE", with_zero


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
def test_zero_and_tiny_densities_match_the_oracle(engine):
    """Zeros and magnitudes below float32's normal range (which the split path takes as
    zero) scattered through the density, and whole rows of them, against the oracle: the
    projection's chunks that hold them go through its checked conversion."""
    w = W.presn(n_r=16, n_theta=32, n_phi=64, L=6)
    rng = np.random.default_rng(7)
    flat = w.rho.reshape(-1)
    idx = rng.choice(flat.size, size=flat.size // 50, replace=False)
    flat[idx[: idx.size // 2]] = 0.0
    flat[idx[idx.size // 2:]] = 1e-300
    w.rho[3, 5, :] = 1e-45   # a whole row below float32's range
    w.rho[4, 7, :] = 0.0     # a whole row of zeros
    w.rho[5, 9, 17:] = 0.0   # a row that ends in zeros
    ref = oracle_solve(w)["phi"]
    phi = gpu_solve(w, "bf16x3", want_moments=False, engine=engine)["phi"]
    err = phi_rel_err(phi, ref)
    print(f"zeros and tiny values, {engine}: phi {err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
@pytest.mark.parametrize("shape,L", [((8, 16, 32), 4), ((64, 32, 64), 8)])
def test_expired_device_wait_reports_timeout_and_the_mesh_recovers(shape, L, engine):
    """Failure detection without a fault: a wait budget of one clock cycle makes the
    bounded pipeline waits of the split kernels run out.  Every block then raises its
    abort flag, lets the copies and MMAs it issued finish, frees its tensor memory and
    exits; mp_mesh_synchronize reports MP_ERR_TIMEOUT.  With the default budget back,
    the same mesh solves correctly again."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=shape[0], n_theta=shape[1], n_phi=shape[2], L=L, r_lo=1e7, r_hi=3e7)
    m = w.mesh
    ref = oracle_solve(w)["phi"]
    rho = torch.from_numpy(w.rho).cuda()
    phi = torch.empty_like(rho)
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh:
        assert mesh.info()["effective_precision"] == 1
        mesh.set_theta_engine(engine)
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.solve()
        mesh.synchronize()
        mesh.set_wait_budget(1)
        for _ in range(2):  # graph replay and the eager (profiled) launches
            mesh.solve()
            with pytest.raises(mpl.MultipoleError) as ei:
                mesh.synchronize()
            assert ei.value.name == "MP_ERR_TIMEOUT"
            mesh.profile(True)
        mesh.profile(False)
        mesh.set_wait_budget(0)
        phi.fill_(0.0)
        mesh.solve()
        mesh.synchronize()
        assert phi_rel_err(phi.cpu().numpy(), ref) <= 1e-6


def test_solve_without_density_is_not_ready():
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=4, n_theta=8, n_phi=16, L=2, materialize=False)
    m = w.mesh
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G) as mesh:
        with pytest.raises(mpl.MultipoleError) as ei:
            mesh.solve()
        assert ei.value.name == "MP_ERR_NOT_READY"


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_graph_replay_equals_eager_launches_and_follows_rebinding(prec):
    """mp_solve replays a captured graph; with profiling on it launches the kernels one by
    one.  Both give identical bits, and binding another density re-captures the graph."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=32, n_theta=32, n_phi=64, L=8)
    w2 = W.presn(n_r=32, n_theta=32, n_phi=64, L=8, seed=7)
    m = w.mesh
    rho = torch.from_numpy(w.rho).cuda()
    rho2 = torch.from_numpy(w2.rho).cuda()
    phi = torch.empty_like(rho)
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.solve()
        mesh.solve()
        mesh.synchronize()
        graph_1 = phi.cpu().numpy()
        mesh.profile(True)
        mesh.solve()
        mesh.synchronize()
        eager_1 = phi.cpu().numpy()
        mesh.profile(False)
        mesh.set_density(rho2)
        mesh.solve()
        mesh.synchronize()
        graph_2 = phi.cpu().numpy()
        mesh.set_density(rho)
        mesh.solve()
        mesh.synchronize()
        graph_1b = phi.cpu().numpy()
    assert np.array_equal(graph_1, eager_1)
    assert np.array_equal(graph_1, graph_1b)
    assert not np.array_equal(graph_1, graph_2)
    assert phi_rel_err(graph_2, gpu_solve(w2, prec, want_moments=False)["phi"]) == 0.0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_host_end_to_end_equals_device_solve(prec):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=32, n_theta=32, n_phi=64, L=8)
    m = w.mesh
    dev = gpu_solve(w, prec, want_moments=False)["phi"]
    rho_h = torch.from_numpy(w.rho).pin_memory()
    phi_h = torch.empty_like(rho_h).pin_memory()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        mesh.solve_host_ptr(rho_h.data_ptr(), phi_h.data_ptr())
    assert np.array_equal(phi_h.numpy(), dev)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_async_host_solves_in_flight_equal_device_solves(prec):
    """Five asynchronous host round trips in flight at once (two staging pairs in
    turn, so pairs are reused while earlier downloads may still run): each output
    equals that density's own device solve, and get_phi returns the last one."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    ws = [W.presn(n_r=32, n_theta=32, n_phi=64, L=8, seed=40 + k) for k in range(5)]
    m = ws[0].mesh
    devs = [gpu_solve(w, prec, want_moments=False)["phi"] for w in ws]
    rhos = [torch.from_numpy(w.rho).pin_memory() for w in ws]
    phis = [torch.full_like(r, np.nan).pin_memory() for r in rhos]
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=prec) as mesh:
        for r, p in zip(rhos, phis):
            mesh.solve_host_ptr_async(r.data_ptr(), p.data_ptr())
        mesh.synchronize()
        last = torch.empty(m.cells, dtype=torch.float64, device="cuda")
        mesh.get_phi(last)
        mesh.synchronize()
        # the synchronous call after asynchronous ones reuses the same pairs
        again = torch.empty_like(rhos[0]).pin_memory()
        mesh.solve_host_ptr(rhos[1].data_ptr(), again.data_ptr())
    for k in range(5):
        assert np.array_equal(phis[k].numpy().ravel(), devs[k].ravel()), k
    assert np.array_equal(last.cpu().numpy(), devs[4].ravel())
    assert np.array_equal(again.numpy().ravel(), devs[1].ravel())


def test_batch_equals_individual_solves():
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    ws = [W.presn(n_r=16, n_theta=32, n_phi=64, L=8, seed=11),
          W.presn(n_r=24, n_theta=16, n_phi=32, L=4, seed=12),
          W.random_small((6, 8, 9), 3, seed=13, r0=0.0, r1=1.0)]
    precs = ["bf16x3", "fp64", "fp64"]
    meshes, outs = [], []
    for w, p in zip(ws, precs):
        m = w.mesh
        mesh = mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision=p)
        rho = torch.from_numpy(w.rho).cuda()
        phi = torch.zeros_like(rho)
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        meshes.append(mesh)
        outs.append((rho, phi))
    b = mpl.Batch(meshes)
    for _ in range(2):
        b.solve()
    meshes[0].synchronize()
    for w, p, (rho, phi) in zip(ws, precs, outs):
        ref = gpu_solve(w, p, want_moments=False)["phi"]
        assert np.array_equal(phi.cpu().numpy(), ref)
    b.close()
    for mesh in meshes:
        mesh.close()


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
def test_profile_names_every_kernel(engine):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=16, n_theta=32, n_phi=64, L=8)
    m = w.mesh
    rho = torch.from_numpy(w.rho).cuda()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh:
        mesh.set_theta_engine(engine)
        mesh.set_density(rho)
        mesh.profile(True)
        for _ in range(3):
            mesh.solve()
        prof = mesh.profile_read()
    theta = {"tensor": ("split_theta_contract_m0", "split_theta_contract_tc", "split_theta_synth_m0",
                        "split_theta_synth_tc"),
             "cuda": ("split_theta_contract", "split_theta_synth")}[engine]
    assert set(prof) == {"split_phi_project_tc", "radial_scan", "split_synth_tc", *theta}
    assert all(v["launches"] == 3 and v["total_ms"] > 0 for v in prof.values())


@pytest.mark.parametrize("shape,L", [((32, 32, 64), 8), ((32, 64, 512), 40)])
def test_every_synthesis_stage_configuration_matches_the_oracle(tmp_path, shape, L):
    """Each stage configuration of the phi synthesis (A stages, table residency or ring,
    staging boxes of 16 or 8 columns), applied through a tuner cache line, against the
    oracle.  Lines that do not fit a mesh's shared memory are not applied (the tuner then
    times candidates instead), and are skipped here.  The radial range keeps neighbouring
    edges within a factor 1.05 (the midpoint split weighs a shell's own degree-l moment by
    (r_{i+1}/r_i)^l, which at l = 40 and a factor 2 would leave no digit to compare)."""
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=shape[0], n_theta=shape[1], n_phi=shape[2], L=L, r_lo=1e7, r_hi=4e7)
    m = w.mesh
    ref = oracle_solve(w)["phi"]
    rho = torch.from_numpy(w.rho).cuda()
    phi = torch.empty_like(rho)
    applied = 0
    for sy in range(12):
        cache = tmp_path / f"tune_{sy}.txt"
        with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh:
            # key (n_r n_theta n_phi l_max precision), then ns_s sy sw br tc gs_ns nacc, format tag
            cache.write_text(f"{shape[0]} {shape[1]} {shape[2]} {L} 1 2 {sy} 128 0 1 8 1 s2\n")
            mesh.set_density(rho)
            mesh.set_phi_output(phi)
            mesh.autotune(str(cache))
            if mesh.info()["tuned_candidates"] != 0:
                continue  # this configuration does not fit the mesh
            applied += 1
            phi.fill_(float("nan"))
            mesh.solve()
            mesh.synchronize()
            err = phi_rel_err(phi.cpu().numpy(), ref)
            assert err <= 1e-6, (sy, err)
    assert applied >= 6, applied


def test_autotune_keeps_results(tmp_path):
    import torch
    from paper_2602_02507_gb300 import multipole as mpl
    w = W.presn(n_r=32, n_theta=32, n_phi=64, L=8)
    m = w.mesh
    ref = oracle_solve(w)["phi"]
    rho = torch.from_numpy(w.rho).cuda()
    phi = torch.empty_like(rho)
    cache = str(tmp_path / "tune.txt")
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh:
        mesh.set_density(rho)
        mesh.set_phi_output(phi)
        mesh.autotune(cache)
        assert mesh.info()["tuned_candidates"] > 1  # configurations were actually timed
        engine = mesh.info()["theta_tensor_cores"]
        mesh.solve()
        mesh.synchronize()
        assert phi_rel_err(phi.cpu().numpy(), ref) <= 1e-6
    assert open(cache).read().strip()
    with mpl.Mesh(m.r, m.theta, m.phi, m.L, m.G, precision="bf16x3") as mesh2:
        mesh2.set_density(rho)
        mesh2.autotune(cache)  # served from the cache
        assert mesh2.info()["tuned_candidates"] == 0
        assert mesh2.info()["theta_tensor_cores"] == engine
