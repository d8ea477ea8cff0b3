"""The allocation-free translation entry point (lsms_translate_mixed_noalloc).

It serves callers that cannot allocate device memory themselves: code whose device memory is owned
by someone else (a framework's pooled allocator, a pre-sized arena) or that runs in a latency-
critical loop where cudaMalloc/cudaFree, which may synchronise the device, are not allowed.  Its
output must match the context entry point lsms_translate(..., LSMS_MIXED) within the tolerance the
mixed-operator parity tests use, on consecutive calls (the scratch array keeps the previous call's
contents, so a second call with other inputs checks that nothing stale leaks through), and the
oracle's pair-by-pair translation on sampled target discs.  The binding refuses tensors of the
wrong type, shape, device or layout before they reach the kernels.

This file is collected after every other test file (pytest --collect-only shows the order): a run
that stops at the first failure has then already run them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_MIXED_OP = 2e-5


def test_noalloc_translation_matches_the_context_entry_point():
    import torch

    import __graft_entry__
    from oracle import lsms_oracle as O
    from paper_1407_3868_gb300 import inputs, lsms

    __graft_entry__.build()
    w = inputs.WORKLOADS["disc1000_p12_ns512"]
    m = w.medium
    centres = w.centres()
    ctx = lsms.context_for(w)
    ctx.set_particles(centres)
    hs = O.order_scale(w.p, m["k2"], m["radius"])
    weight = hs * np.abs(O.mie_coefficients(w.p, m["k2"], m["kp"], m["radius"]))
    c_dev = torch.from_numpy(np.ascontiguousarray(centres)).cuda()
    for seed in (31, 32):
        beta = inputs.random_coefficients(w.n, w.p, 2, seed) / hs
        ref = ctx.translate(beta, precision=lsms.LSMS_MIXED)
        b_dev = torch.from_numpy(beta).cuda()
        a_dev = torch.full_like(b_dev, complex(float("nan"), float("nan")))
        lsms.translate_mixed_noalloc(c_dev, b_dev, a_dev, m["k2"], w.p)
        torch.cuda.synchronize()
        got = a_dev.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.linalg.norm((got - ref) * weight) / np.linalg.norm(ref * weight)
        assert err < TOL_MIXED_OP, (seed, err)
        # and against the oracle's translation (Lemma 3.1 summed pair by pair) on sampled targets,
        # element by element in the weighted norm
        rows = sorted(set([0, w.n - 1] + list(np.random.default_rng(seed).choice(w.n, 6, replace=False))))
        for r in range(2):
            a_o = O.translate(centres, beta[r], m["k2"], w.p, rows)
            e_max = np.max(np.abs((got[r][rows] - a_o) * weight)) / np.max(np.abs(a_o * weight))
            assert e_max < TOL_MIXED_OP, (seed, r, e_max)
    ctx.close()


def test_noalloc_translation_checks_its_tensors():
    import torch

    from paper_1407_3868_gb300 import lsms

    n, p = 8, 3
    c = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    b = torch.zeros((1, n, 2 * p + 1), dtype=torch.complex128, device="cuda")
    bad = [
        (c.float(), b, b),                                   # centres not float64
        (c, b.to(torch.complex64), b),                       # beta not complex128
        (c, b, b[:, :4]),                                    # alpha smaller than beta
        (c, b[:, :, :5], b[:, :, :5]),                       # not nrhs x n x (2p+1)
        (c.cpu(), b, b),                                     # host tensor
        (c, b, b.transpose(1, 2)),                           # not contiguous
        (c.reshape(-1), b, b),                               # centres not (n, 2)
    ]
    for args in bad:
        with pytest.raises(ValueError):
            lsms.translate_mixed_noalloc(*args, 3.0, p)


def test_noalloc_translation_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_1407_3868_gb300 import lsms

    n, p = 40000, 14                      # 16 n + 16 n (2p+1) bytes > 16 MiB
    c = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    b = torch.zeros((1, n, 2 * p + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(lsms.LsmsError) as e:
        lsms.translate_mixed_noalloc(c, b, b, 3.0, p)
    assert e.value.code == -1
    assert "16 MiB" in str(e.value)
