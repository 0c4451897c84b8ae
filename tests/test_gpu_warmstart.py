"""GPU checks of the learned warm start (tomo_ws_*) against the FP64 oracle
network, and of what the trained network gains in the solve."""
import numpy as np
import pytest

from conftest import small_cfg
from oracle import cnn
from oracle import geometry as geo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_07938_gb300 import tomo
    tomo.lib()
    return tomo


def init_params(NP, hidden, seed, last_gain=0.1, cin=None):
    rng = np.random.default_rng(seed)
    out = []
    shapes = cnn.layer_shapes(NP, hidden)
    if cin is not None:
        shapes[0] = (hidden, cin)
    for l, (co, ci) in enumerate(shapes):
        W = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        if l == 3:
            W *= last_gain
        out += [W.ravel(), 0.01 * rng.standard_normal(co)]
    return np.concatenate(out).astype(np.float32)


@pytest.mark.parametrize("n,hidden,B,hybrid", [(7, 5, 3, False), (7, 5, 3, True), (74, 32, 2, False)])
def test_forward_and_gradient_match_oracle(T, n, hidden, B, hybrid):
    from oracle import precond
    cfg = small_cfg(n=n, n_gs=2 if n < 20 else 6, lgs=True, obstruction=0.2 if n < 20 else 0.28, D=0.527 * n)
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B, precond=hybrid)
    try:
        info, _, _ = T.tomo_layout(h)
        NP = 2 * len(cfg["gs"])
        T.tomo_ws_init(h, hidden=hidden, max_batch=B, in_scale=0.5, out_scale=2.0, precond_input=hybrid, pre_gain=0.7)
        params = init_params(NP, hidden, seed=n, last_gain=1.0, cin=2 * NP if hybrid else None)
        T.tomo_ws_set_params(h, params)
        assert np.array_equal(T.tomo_ws_get_params(h), params)
        rng = np.random.default_rng(1)
        s = rng.standard_normal((B, info.N)).astype(np.float32)
        t = rng.standard_normal((B, info.N)).astype(np.float32)
        sd = torch.tensor(s, device="cuda")
        td = torch.tensor(t, device="cuda")
        z = torch.empty_like(sd)
        T.tomo_ws_apply(h, sd, z, B)
        torch.cuda.synchronize()
        pre = precond.apply(cfg, s, info.P) if hybrid else None
        z_ref, _ = cnn.forward(params.astype(np.float64), s, n, cfg["obstruction"], hidden, 0.5, 2.0, pre, 0.7)
        zg = z.double().cpu().numpy()
        assert np.linalg.norm(zg - z_ref) / np.linalg.norm(z_ref) <= 1e-5
        g, loss = T.tomo_ws_gradient(h, sd, td, B)
        loss_ref, g_ref = cnn.loss_and_grad(params.astype(np.float64), s, t, n, cfg["obstruction"], hidden, 0.5, 2.0,
                                            pre, 0.7)
        assert abs(loss - loss_ref) <= 1e-5 * loss_ref
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-4
    finally:
        T.tomo_destroy(h)


def test_adam_steps_match_oracle(T):
    # tomo_ws_train_step is the gradient (checked above) followed by one Adam
    # step (Kingma & Ba 2015): two steps in a row, each against
    # oracle.cnn.adam_step applied to the same gradient, the oracle carrying
    # its own moment estimates from step to step
    cfg = small_cfg(n=7, n_gs=2, lgs=True, obstruction=0.2, D=0.527 * 7)
    B, hidden, lr = 3, 5, 1e-2
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B)
    try:
        info, _, _ = T.tomo_layout(h)
        T.tomo_ws_init(h, hidden=hidden, max_batch=B, in_scale=0.5, out_scale=2.0)
        T.tomo_ws_set_params(h, init_params(4, hidden, seed=3, last_gain=1.0))   # also resets m, v and t
        rng = np.random.default_rng(8)
        m = v = 0.0
        for t in (1, 2):
            sd = torch.tensor(rng.standard_normal((B, info.N)).astype(np.float32), device="cuda")
            td = torch.tensor(rng.standard_normal((B, info.N)).astype(np.float32), device="cuda")
            p_prev = T.tomo_ws_get_params(h).astype(np.float64)
            g, _ = T.tomo_ws_gradient(h, sd, td, B)           # the gradient the step uses (no update)
            p_exp, m, v = cnn.adam_step(p_prev, g, m, v, t, lr)
            T.tomo_ws_train_step(h, sd, td, B, lr)
            p = T.tomo_ws_get_params(h).astype(np.float64)
            # every parameter within 1e-5 of the oracle's (the steps are about
            # lr = 1e-2 each, so this is 1e-3 of a step)
            print("adam step", t, "max |p - p_oracle|", np.abs(p - p_exp).max())
            assert np.abs(p - p_exp).max() <= 1e-5
            assert np.abs(p - p_prev).max() > 0.5 * lr
    finally:
        T.tomo_destroy(h)


def test_training_gains_iterations(T):
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("lgs_mid")
    n_train, n_test = 256, 32
    full, sigma = W.slope_frames(cfg, n_train + n_test, seed=7)
    cfg["noise_sigma"] = [float(x) for x in sigma]
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    s = full[..., mask].reshape(n_train + n_test, -1).astype(np.float32)
    B = 32
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B, precond=True)
    try:
        sd = torch.tensor(s, device="cuda")
        zs = torch.zeros_like(sd)
        for b0 in range(0, n_train + n_test, B):
            T.tomo_solve(h, sd[b0:b0 + B].contiguous(), B, T.solve_opts(tol=1e-5, precond=True), zs[b0:b0 + B])
        z_np = zs.cpu().numpy()
        NP = 2 * len(cfg["gs"])
        T.tomo_ws_init(h, hidden=32, max_batch=B, in_scale=float(1.0 / s.std()), out_scale=float(z_np.std()))
        T.tomo_ws_set_params(h, init_params(NP, 32, seed=11))
        rng = np.random.default_rng(5)
        losses = []
        for step in range(600):
            idx = rng.choice(n_train, B, replace=False)
            xb = sd[idx].contiguous()
            tb = zs[idx].contiguous()
            losses.append(T.tomo_ws_train_step(h, xb, tb, B, 2e-3 if step < 400 else 5e-4))
        print('loss first/last', np.mean(losses[:10]), np.mean(losses[-50:]))
        assert np.mean(losses[-50:]) < 0.85 * np.mean(losses[:10])
        # held-out frames: warm start from the network vs cold start
        st = sd[n_train:].contiguous()
        z0 = torch.empty_like(st)
        T.tomo_ws_apply(h, st, z0, n_test)
        zt = zs[n_train:].cpu().numpy()
        rel = np.linalg.norm(z0.cpu().numpy() - zt) / np.linalg.norm(zt)
        zc = torch.zeros_like(st)
        cold = T.tomo_solve(h, st, n_test, T.solve_opts(tol=1e-4, precond=True), zc)
        zw = torch.zeros_like(st)
        warm = T.tomo_solve(h, st, n_test, T.solve_opts(tol=1e-4, precond=True, warm_start=2), zw)
        print(f"warm start: held-out relative error {rel:.3f}; PCG iterations cold {cold['iters'].mean():.1f} "
              f"warm {warm['iters'].mean():.1f}; final loss {np.mean(losses[-50:]):.3f}")
        assert (warm["status"] == 0).all() and (warm["relres"] <= 1e-4).all()
        assert rel < 1.0
        assert warm["iters"].mean() < cold["iters"].mean()
    finally:
        T.tomo_destroy(h)


# --------------------------------------------------------------------------- learned flexible PCG
def _lgs_mid_frames(T, n, seed):
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("lgs_mid")
    full, sigma = W.slope_frames(cfg, n, seed=seed)
    cfg["noise_sigma"] = [float(x) for x in sigma]
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    return cfg, full[..., mask].reshape(n, -1).astype(np.float32)


def _bound_ok(cfg, s, z, info):
    from oracle import covariance as cov
    from oracle import solve
    A = cov.system_matrix(cfg)
    zs = solve.solve_cholesky(A, s.astype(np.float64).T).T
    bound = info["relres"] * np.linalg.norm(s, axis=1) / min(cfg["noise_sigma"]) ** 2
    return (np.linalg.norm(z - zs, axis=1) <= bound).all()


def test_flexible_pcg_zero_network_is_pcg_and_bad_network_falls_back(T):
    # with a zero network the learned preconditioner is M itself: flexible
    # PCG is then PCG with M in its textbook form (Polak-Ribiere beta equals
    # the standard one for a fixed M in exact arithmetic); it must converge
    # without falling back and in no more iterations than the library's PCG
    # (Chronopoulos-Gear form, whose FP32 recurrences cost iterations: 540-593
    # here against 428-479 measured).  A network whose output is no descent
    # direction makes every frame fall back to PCG with M, which still
    # converges to the oracle's solution (TOMO_FRAME_FALLBACK_PLAIN_CG)
    cfg, s = _lgs_mid_frames(T, 4, seed=40)
    B = 4
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B, precond=True)
    try:
        sd = torch.tensor(s, device="cuda")
        zp = torch.zeros_like(sd)
        pcg = T.tomo_solve(h, sd, B, T.solve_opts(tol=1e-5, max_iter=20000, max_refine=3, precond=True), zp)
        T.tomo_ws_init(h, hidden=8, max_batch=B, in_scale=1.0, out_scale=1.0, precond_input=True, pre_gain=1.0)
        zf = torch.zeros_like(sd)
        flex = T.tomo_solve(h, sd, B, T.solve_opts(tol=1e-5, max_iter=20000, max_refine=3, precond="learned"), zf)
        print("PCG", pcg["iters"], "flexible, zero network", flex["iters"], flex["status"])
        assert (flex["status"] == T.FRAME_CONVERGED).all() and (flex["relres"] <= 1e-5).all()
        assert (flex["iters"] <= 1.1 * pcg["iters"]).all()
        assert _bound_ok(cfg, s, zf.double().cpu().numpy(), flex)
        # a harmful network: no M term, large random weights
        n_par = T.tomo_ws_param_count(h)
        rng = np.random.default_rng(3)
        h2 = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B, precond=True)
        try:
            T.tomo_ws_init(h2, hidden=8, max_batch=B, in_scale=1.0, out_scale=1.0, precond_input=True, pre_gain=0.0)
            T.tomo_ws_set_params(h2, (rng.standard_normal(n_par) * 3.0).astype(np.float32))
            zb = torch.zeros_like(sd)
            bad = T.tomo_solve(h2, sd, B, T.solve_opts(tol=1e-5, max_iter=20000, max_refine=3, precond="learned"), zb)
            print("flexible, harmful network", bad["iters"], bad["status"])
            assert (bad["status"] == T.FRAME_FALLBACK_PLAIN_CG).all() and (bad["relres"] <= 1e-5).all()
            assert _bound_ok(cfg, s, zb.double().cpu().numpy(), bad)
        finally:
            T.tomo_destroy(h2)
        # the learned preconditioner needs the [r, M r] network and method CG
        with pytest.raises(T.TomoError):
            T.tomo_solve(h, sd, B, T.solve_opts(precond="learned", method="minres"), zf)
    finally:
        T.tomo_destroy(h)


def residual_pairs(T, h, sd, zstar, B, ks):
    """(r_k, zeta* - x_k) of truncated PCG solves (x_k after k iterations), each
    pair scaled to |r_k| = 1: the residuals the preconditioner meets and the
    errors A^{-1} r_k it should approximate."""
    rs, es = [], []
    for k in ks:
        x = torch.zeros_like(sd)
        if k > 0:
            T.tomo_solve(h, sd, B, T.solve_opts(tol=1e-12, max_iter=k, max_refine=0, check_every=1, precond=True), x)
        Ax = torch.empty_like(sd)
        T.tomo_apply_css(h, x, Ax, B)
        r = sd - Ax
        e = zstar - x
        nr = r.norm(dim=1, keepdim=True)
        rs.append(r / nr)
        es.append(e / nr)
    return torch.cat(rs).contiguous(), torch.cat(es).contiguous()


def test_learned_flexible_pcg_gain(T):
    # the learned preconditioner trained on (residual, error) pairs of
    # truncated PCG solves of training frames, then used in flexible PCG on
    # held-out frames: the gain over PCG with M alone is stated (it may be
    # negative); every frame converges to the oracle's solution either way
    cfg, s = _lgs_mid_frames(T, 96, seed=41)
    n_train, n_test, B = 64, 32, 32
    h = T.tomo_create(cfg, stream=torch.cuda.current_stream(), max_batch=B, precond=True)
    try:
        sd = torch.tensor(s, device="cuda")
        zs = torch.zeros_like(sd)
        for b0 in range(0, n_train + n_test, B):
            T.tomo_solve(h, sd[b0:b0 + B].contiguous(), B, T.solve_opts(tol=1e-6, max_iter=30000, precond=True),
                         zs[b0:b0 + B])
        rp, ep = [], []
        for b0 in range(0, n_train, B):
            r, e = residual_pairs(T, h, sd[b0:b0 + B].contiguous(), zs[b0:b0 + B].contiguous(), B, (0, 8, 30, 80))
            rp.append(r)
            ep.append(e)
        rp, ep = torch.cat(rp), torch.cat(ep)
        NP = 2 * len(cfg["gs"])
        T.tomo_ws_init(h, hidden=16, max_batch=B, in_scale=float(1.0 / rp.std()), out_scale=float(ep.std()),
                       precond_input=True, pre_gain=1.0)
        T.tomo_ws_set_params(h, init_params(NP, 16, seed=12, last_gain=0.0, cin=2 * NP))
        rng = np.random.default_rng(6)
        losses = []
        for step in range(400):
            idx = torch.tensor(rng.choice(rp.shape[0], B, replace=False), device="cuda")
            losses.append(T.tomo_ws_train_step(h, rp[idx].contiguous(), ep[idx].contiguous(), B,
                                               1e-3 if step < 300 else 3e-4))
        st = sd[n_train:].contiguous()
        out = {}
        for name, pc in (("pcg", True), ("learned", "learned")):
            z = torch.zeros_like(st)
            T.tomo_solve(h, st, n_test, T.solve_opts(tol=1e-4, max_iter=30000, precond=pc), z)   # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = T.tomo_solve(h, st, n_test, T.solve_opts(tol=1e-4, max_iter=30000, precond=pc), z)
            e1.record()
            torch.cuda.synchronize()
            out[name] = (info, e0.elapsed_time(e1), z.double().cpu().numpy())
        ip, tp, _ = out["pcg"]
        il, tl, zl = out["learned"]
        print(f"learned flexible PCG: loss {np.mean(losses[:10]):.3f} -> {np.mean(losses[-50:]):.3f}; "
              f"iterations PCG {ip['iters'].mean():.1f} learned {il['iters'].mean():.1f} "
              f"(gain {1 - il['iters'].mean() / ip['iters'].mean():+.1%}); time PCG {tp:.1f} ms learned {tl:.1f} ms "
              f"(frames/s gain {tp / tl - 1:+.1%}); fallbacks {(il['status'] == T.FRAME_FALLBACK_PLAIN_CG).sum()}")
        assert np.isin(il["status"], [T.FRAME_CONVERGED, T.FRAME_FALLBACK_PLAIN_CG]).all()
        assert (il["relres"] <= 1e-4).all()
        assert _bound_ok(cfg, s[n_train:], zl, il)
    finally:
        T.tomo_destroy(h)
