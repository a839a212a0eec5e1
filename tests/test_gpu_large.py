"""Parity at the full sizes of the 128^3 and 512^3 workloads, in the launch
configuration the benchmark times (n_sub = 2, B-spline softening)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2112_01508_gb300 import ShortRange
from tests._gpu_helpers import gpu_forces, rel_rms

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_n2m_full_parity():
    w = synth.workload("n2m")
    pos = synth.workload_positions(w)
    ref, pairs = oracle.sr_accel(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
    r64 = gpu_forces(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps, precision=64, n_sub=w.n_sub)
    assert r64["pairs"] == pairs
    e64 = rel_rms(r64["acc"], ref)
    r32 = gpu_forces(pos, w.x_s, w.x_r, w.G_m, "bspline", w.eps, precision=32, n_sub=w.n_sub)
    e32 = rel_rms(r32["acc"], ref)
    print(f"n2m: pairs {pairs} fp64 rel RMS {e64:.3e} fp32 rel RMS {e32:.3e} fp32 pairs {r32['pairs']}")
    assert e64 <= 1e-12
    assert e32 <= 1e-5
    assert abs(r32["pairs"] - pairs) <= 1e-6 * pairs


def test_n2m_mesh_parity():
    """The long-range mesh force of the benchmark set (128^3 particles, 256^3 mesh, CIC,
    D_4) against the PM oracle: full density and potential, accelerations compared on
    a seeded sample of 2^16 particles."""
    import torch

    from oracle import pm as opm
    from paper_2112_01508_gb300 import LongRange

    w = synth.workload("n2m")
    pos = synth.workload_positions(w)
    idx = np.sort(np.random.default_rng(3).choice(w.n, 1 << 16, replace=False))
    phi = opm.potential_mesh(opm.assign(pos, w.n_phi, 2), w.x_s, 2)
    ref = np.empty((3, len(idx)))
    for d in range(3):
        ref[d] = opm.interpolate(opm.difference(phi, 4, d), pos[:, idx], 2)
    ref *= 4 * np.pi * w.G_m * w.n_phi ** 4
    p = torch.from_numpy(pos).cuda()
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        with LongRange.from_workload(w, precision=prec) as lr:
            a = lr.accel(p)
            lr.sync()
            got = a.double().cpu().numpy()[:, idx]
        err = rel_rms(got, ref)
        print(f"n2m mesh fp{prec}: rel RMS {err:.3e} over {len(idx)} particles")
        assert err <= tol


def test_n134m_sampled_with_rungs():
    """512^3: rungs from the FP64 fake kick (bit-exact vs the oracle's rule on the
    same accelerations), then the FP32 and FP64 forces of the active rungs on
    2^18 sampled receivers against the oracle."""
    w = synth.workload("n134m")
    n = w.n
    pos = synth.workload_positions(w)
    dev = torch.device("cuda")
    eta = 0.025
    with ShortRange.from_workload(w) as sr:
        p = torch.from_numpy(pos).to(dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        sr.sort(p, perm_out=perm)
        sr.build_pairs()
        a64 = sr.forces(p, 64)
        amag = torch.linalg.vector_norm(a64, dim=0)
        sample = torch.randperm(n, device=dev, generator=torch.Generator(device=dev).manual_seed(0))[:1 << 20]
        q99 = float(torch.quantile(amag[sample].float(), 0.99))
        dt = 64.0 * (2.0 * eta * w.eps / q99) ** 0.5
        rung = sr.assign_rungs(a64, dt, eta, w.eps)
        sr.sync()
        perm_np = perm.cpu().numpy().astype(np.int64)
        rung_np = rung.cpu().numpy()
        rng = np.random.default_rng(5)
        check = rng.choice(n, size=1 << 18, replace=False)
        a64_np = a64[:, torch.from_numpy(check).to(dev)].cpu().numpy()
        ref_r, _ = oracle.rungs(a64_np, dt, eta, w.eps, 8)
        np.testing.assert_array_equal(rung_np[check], ref_r)
        hist = np.bincount(rung_np, minlength=8)
        print("rung histogram", hist)
        assert hist[7] > 0.005 * n
        pos_sorted = p.cpu().numpy()
        for rung_min in (0, 5, 7):
            sr.build_pairs(rung, rung_min)
            out32 = torch.full((3, n), float("nan"), dtype=torch.float32, device=dev)
            sr.forces(p, 32, out32)
            out64 = sr.forces(p, 64)
            st = sr.stats()
            act = np.nonzero(rung_np >= rung_min)[0]
            recv = np.sort(rng.choice(act, size=min(1 << 18, len(act)), replace=False))
            ref, _ = oracle.sr_accel_subset(pos_sorted, recv, w.x_s, w.x_r, w.G_m, "bspline", w.eps)
            ridx = torch.from_numpy(recv).to(dev)
            g32 = out32[:, ridx].cpu().numpy()
            g64 = out64[:, ridx].cpu().numpy()
            e32, e64 = rel_rms(g32, ref), rel_rms(g64, ref)
            print(f"n134m rung_min={rung_min}: active {st.n_active} fp32 {e32:.3e} fp64 {e64:.3e}")
            assert st.n_active == len(act)
            assert e64 <= 1e-12
            assert e32 <= 1e-5
            inact = np.nonzero(rung_np < rung_min)[0]
            if len(inact):
                probe = torch.from_numpy(inact[:4096]).to(dev)
                assert torch.isnan(out32[:, probe]).all()


def test_n1g_sampled():
    """1024^3: the FP32 forces of all particles, and the FP64 forces of the deepest
    rung (~1% active), on 2^18 sampled receivers against the oracle; rungs
    bit-exact on the sample."""
    w = synth.workload("n1g")
    n = w.n
    pos = synth.workload_positions(w)
    dev = torch.device("cuda")
    eta = 0.025
    rng = np.random.default_rng(11)
    with ShortRange.from_workload(w) as sr:
        p = torch.from_numpy(pos).to(dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        sr.sort(p, perm_out=perm)
        sr.build_pairs()
        a32 = sr.forces(p, 32)
        st = sr.stats()
        print(f"n1g: {st.pairs_last} interacting pairs, FP32 kernel {st.force_kernel_ms:.1f} ms")
        amag = torch.linalg.vector_norm(a32, dim=0)
        sample = torch.randperm(n, device=dev, generator=torch.Generator(device=dev).manual_seed(0))[:1 << 20]
        q99 = float(torch.quantile(amag[sample], 0.99))
        del amag
        dt = 64.0 * (2.0 * eta * w.eps / q99) ** 0.5
        rung = sr.assign_rungs(a32, dt, eta, w.eps)
        k32 = np.sort(rng.choice(n, size=1 << 18, replace=False))
        kk = torch.from_numpy(k32).to(dev)
        g32 = a32[:, kk].cpu().numpy()
        ref_r, _ = oracle.rungs(g32.astype(np.float64), dt, eta, w.eps, 8)
        np.testing.assert_array_equal(rung[kk].cpu().numpy(), ref_r)
        sr.build_pairs(rung, 7)
        a64 = torch.full((3, n), float("nan"), dtype=torch.float64, device=dev)
        sr.forces(p, 64, a64)
        st = sr.stats()
        act = torch.nonzero(rung >= 7).flatten()
        k64 = act[torch.randperm(len(act), device=dev, generator=torch.Generator(device=dev).manual_seed(1))[:1 << 18]]
        k64 = torch.sort(k64).values
        g64 = a64[:, k64].cpu().numpy()
        perm_np = perm.cpu().numpy().astype(np.int64)
        assert st.n_active == len(act)
    del p
    for name, ks, got, tol in (("fp32", k32, g32, 1e-5), ("fp64 rung 7", k64.cpu().numpy(), g64, 1e-12)):
        ref, _ = oracle.sr_accel_subset(pos, perm_np[ks], w.x_s, w.x_r, w.G_m, "bspline", w.eps)
        err = rel_rms(got, ref)
        print(f"n1g {name}: rel RMS {err:.3e} over {len(ks)} receivers")
        assert err <= tol
