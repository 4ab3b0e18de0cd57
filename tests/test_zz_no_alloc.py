"""sn_moment_noalloc: the context-free moment for callers that cannot allocate device memory
(they only hold device buffers owned by a host framework's allocator, or must avoid the
device-wide synchronisation of cudaMalloc/cudaFree).  Checked through the C ABI against the
context's sn_moment on two calls in a row; this file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_noalloc_moment_matches_context_moment_twice():
    import sn_inputs as si
    import paper_1810_11080_gb300 as g
    from paper_1810_11080_gb300._lib import sn_moment_noalloc

    prob = si.make_config("2d_smooth_q3_p3_s8", n=9)
    stream = torch.cuda.Stream()
    ctx = g.setup_problem(prob, device=0, stream=stream.cuda_stream)
    ctx.sn_build_graph("face", 10)
    E, N, M = prob.mesh.n_elem, (prob.p + 1) ** 2, len(prob.w)
    rng = np.random.default_rng(77)
    with torch.cuda.stream(stream):
        w = torch.from_numpy(np.ascontiguousarray(prob.w)).cuda()
        phi_prev = torch.from_numpy(rng.uniform(0.5, 2.0, size=(E, N))).cuda()
    stream.synchronize()
    for call in range(2):
        with torch.cuda.stream(stream):
            psi = torch.from_numpy(rng.uniform(0.0, 1.0 + call, size=(M, E, N))).cuda()
            ref = torch.zeros((E, N), dtype=torch.float64, device="cuda")
            out = torch.full((E, N), float("nan"), dtype=torch.float64, device="cuda")
        stream.synchronize()
        r_ref = ctx.sn_moment(psi, phi_prev, ref)
        r_new = sn_moment_noalloc(0, stream.cuda_stream, w, psi, phi_prev, out)
        stream.synchronize()
        err = torch.linalg.norm(out - ref).item() / torch.linalg.norm(ref).item()
        assert err <= 1e-14, (call, err)
        assert abs(r_new - r_ref) <= 1e-14 * max(abs(r_ref), 1.0), (call, r_new, r_ref)
        phi_prev = out.clone()


def test_noalloc_moment_rejects_sizes_beyond_its_scratch():
    import paper_1810_11080_gb300 as g
    lib = g.lib()
    big_elem = 4194304 // 16 + 1
    st = lib.sn_moment_noalloc(0, None, 4, big_elem, 16, None, None, None, None, None)
    assert st == 1      # SN_EINVAL, before touching any pointer


def test_noalloc_moment_rejects_host_buffers_and_keeps_the_current_device():
    import ctypes
    import paper_1810_11080_gb300 as g
    lib = g.lib()
    before = torch.cuda.current_device()
    E, N, M = 8, 4, 3
    w = torch.ones(M, dtype=torch.float64, device="cuda")
    psi_host = np.ones((M, E, N))
    out = torch.zeros((E, N), dtype=torch.float64, device="cuda")
    st = lib.sn_moment_noalloc(0, None, M, E, N, ctypes.c_void_p(w.data_ptr()),
                               psi_host.ctypes.data_as(ctypes.c_void_p), None,
                               ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1      # SN_EINVAL: psi is host memory, nothing is staged
    assert torch.cuda.current_device() == before
