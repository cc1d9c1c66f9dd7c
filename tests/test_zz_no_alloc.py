"""The allocation-free entry point dd_execute_noalloc, called through the C
ABI, gives exactly the sums of dd_execute, on two calls in a row with
different bands, DM lists and gulps (so nothing left in its shared scratch
array from the first call leaks into the second), and refuses a band whose
tables do not fit its fixed scratch array.

It exists for callers that cannot allocate device memory: real-time loops
where cudaMalloc/cudaFree would stall or synchronise the device, and hosts
that own all device memory through their own pool.  This file is collected
last so that a run stopping at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc(L, f, dms, d_in, nsamp, out):
    import torch

    f = np.ascontiguousarray(f, np.float64)
    dms = np.ascontiguousarray(dms, np.float64)
    st = L.dd_execute_noalloc(f.size, f.ctypes.data, 64e-6, dms.size, dms.ctypes.data,
                              ctypes.c_void_p(d_in.data_ptr()), d_in.stride(0), nsamp,
                              ctypes.c_void_p(out.data_ptr()), out.stride(0),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_matches_dd_execute_twice():
    import torch

    import oracle
    import paper_1112_0065_gb300 as P

    L = P.load_library()
    cases = [
        # band, DMs, gulp: the 1024-channel x 1500-trial single-beam shape (2^17 samples) ...
        (synth.band_freqs(1024), synth.dm_list_piecewise(1000.0), (1 << 17), synth.BASE_SEED + 71),
        # ... then a different, smaller and ragged one
        (synth.band_freqs(130), synth.dm_list_linear(37, 90.0), 9999, synth.BASE_SEED + 72),
    ]
    runs = []
    for f, dms, nout_target, seed in cases:
        plan = P.Plan(f, 64e-6, dms)
        nsamp = nout_target + plan.maxdelay
        d_in = synth.device_noise_packed(f.size, nsamp, seed=seed)
        want = plan.execute(d_in, nsamp)
        got = plan.alloc_output(nsamp)
        got.fill_(-7)
        runs.append((f, dms, nsamp, d_in, want, got, plan.nout(nsamp)))
        torch.cuda.synchronize()
        plan.close()
    # both calls back to back on one stream, no host synchronisation between
    # them: the second rebuilds the host-side tables while the first may still
    # be running
    for f, dms, nsamp, d_in, _, got, _ in runs:
        assert _noalloc(L, f, dms, d_in, nsamp, got) == 0, L.dd_last_error()
    torch.cuda.synchronize()
    for f, dms, nsamp, d_in, want, got, n in runs:
        assert torch.equal(got[:, :n], want[:, :n])
    # the small case also against the CPU oracle's sums
    f, dms, nsamp, d_in, _, got, n = runs[1]
    ref = oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), d_in.cpu().numpy(), nsamp)
    np.testing.assert_array_equal(P.as_uint32(got[:, :n]), ref)


def test_noalloc_rejects_tables_beyond_scratch():
    import torch

    import paper_1112_0065_gb300 as P

    L = P.load_library()
    f = synth.band_freqs(2048)
    dms = synth.dm_list_linear(1100, 5.0)  # 2048 x 1100 x 4 bytes > 8 MiB
    d_in = torch.zeros((2048, 1024), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1100, 4096), dtype=torch.int32, device="cuda")
    assert _noalloc(L, f, dms, d_in, 4000, out) == P._lib.DD_ERR_INVALID_ARG
    assert b"scratch" in L.dd_last_error()
