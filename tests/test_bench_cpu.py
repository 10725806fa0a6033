"""Host logic of bench.py and of the stream generator, checked on the CPU.

The launch-count mirror (`svd_launch_groups`, `LEARNED_FIXED_LAUNCHES`) must agree with what
the GPU ran: an ncu launch list of the learned batched prox on the 512-tensor batch showed
22 kernel launches per call with one DFT launch per direction, 10 of them `svd_kernel` over two
calls (5 Jacobi launch groups at the default CTA shape), and a bench run under the autotuned
shape (target 7, 32 warps, shared launches) reported 210 launches over 10 steps, i.e. 4 Jacobi
groups.  The DFTs of mixed lengths now launch once per register class (two classes in this
batch) and the sketch has a fifth (global-scratch) class launch, 25 launches per call.
"""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1806_07247_gb300 import synth  # noqa: E402


def _batch_shapes():
    return [(s.n1, s.n2) for s in synth.batched_specs(512, 0)]


def test_fixed_launches_of_a_learned_call():
    # features, MLP, binning, 5 class launches, 4 x (collect + retry)
    assert bench.LEARNED_FIXED_LAUNCHES == 16


def test_dft_launch_mirror_matches_the_library_source():
    # the register-class masks mirrored in bench.py are the ones the DFT source defines
    import re
    src = open(os.path.join(ROOT, "paper_1806_07247_gb300", "csrc", "tp_fft.cu")).read()
    m = re.search(r"kClassAtLeast1 = (0x[0-9a-f]+)ull, kClass2 = (0x[0-9a-f]+)ull", src)
    assert m, "class masks not found"
    assert (int(m.group(1), 16), int(m.group(2), 16)) == (bench.DFT_CLASS_AT_LEAST_1,
                                                          bench.DFT_CLASS_2)
    # the batched workload (n3 in 4..64) has lengths of both classes 0 and 1
    n3s = [s.n3 for s in synth.batched_specs(512, 0)]
    assert bench.dft_launches(n3s) == 2
    assert bench.dft_launches([64]) == 1 and bench.dft_launches([64, 64]) == 1
    assert bench.dft_launches([100, 3]) == 1 and bench.dft_launches([5]) == 1


def test_jacobi_groups_match_the_measured_launch_lists():
    shapes = _batch_shapes()
    assert bench.svd_launch_groups(shapes) == 5
    n3s = [s.n3 for s in synth.batched_specs(512, 0)]
    assert bench.LEARNED_FIXED_LAUNCHES + 2 * bench.dft_launches(n3s) + \
        bench.svd_launch_groups(shapes) == 25
    tuned = {"target_lane_pairs": 7, "max_warps": 32, "split_launches": 0}
    assert bench.svd_launch_groups(shapes, tuned) == 4


def test_split_launches_never_merge_fewer_groups():
    shapes = _batch_shapes()
    for e2 in (3, 5, 7):
        for w in (8, 16, 32):
            merged = bench.svd_launch_groups(shapes, {"target_lane_pairs": e2, "max_warps": w,
                                                      "split_launches": 0})
            split = bench.svd_launch_groups(shapes, {"target_lane_pairs": e2, "max_warps": w,
                                                     "split_launches": 1})
            assert split >= merged >= 1


def test_stream_specs_are_seeded_and_in_range():
    a = synth.stream_specs(300, 0)
    assert a == synth.stream_specs(300, 0)
    assert a != synth.stream_specs(300, 1)
    ops = [c.op for c in a]
    assert set(ops) == {"prox", "tprod"}
    assert 0.35 < ops.count("prox") / len(ops) < 0.65
    for c in a:
        for sp in (c.a, c.b) if c.b else (c.a,):
            assert 16 <= sp.n1 <= 512 and 16 <= sp.n2 <= 512
            assert 4 <= sp.n3 <= 256 and 4 <= sp.r <= 40 and sp.noise == 0.02
            nu = 0.02 * math.sqrt(sp.n3) * (math.sqrt(sp.n1) + math.sqrt(sp.n2))
            assert math.isclose(sp.tau, 2.0 * nu, rel_tol=1e-12)
        if c.op == "tprod":
            assert c.b.n1 == c.a.n2 and c.b.n3 == c.a.n3
        else:
            assert c.b is None


def test_job_throughput_is_weak_scaling_units_over_time():
    # 9,359 slices per step, 10 steps in 72.3 ms -> 1.294M slices/s
    assert math.isclose(bench.job_throughput(9359, 10, 72.3), 9359 * 10 / 0.0723)


def test_tprod_oracle_sample_and_sampled_error_on_a_column_major_tensor():
    # the bench's full-size tprod error: sampled Eq. 9 entries against a result laid out as
    # the library lays it out (column-major n1 x l x n3)
    import numpy as np
    import torch

    from oracle import tproduct as O
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.standard_normal((40, 24, 6)).astype(np.float32)
    B = rng.standard_normal((24, 30, 6)).astype(np.float32)
    o = bench.tprod_oracle_sample(A, B, 0.05)
    assert o["literal"]["entries"] >= 64 and o["literal"]["extrapolated_s"] > 0
    assert o["dft_domain"]["block"] == [40, 24, 30, 6] and o["dft_domain"]["extrapolated_s"] > 0
    C = O.tprod(A, B)
    Ct = torch.from_numpy(np.ascontiguousarray(C.transpose(2, 1, 0))).permute(2, 1, 0)
    assert Ct.stride() == (1, 40, 40 * 30)
    assert bench.sampled_rel_err(Ct, o) < 1e-14
    # a wrong entry is seen
    i, l, k = o["idx"][0]
    Ct[i, l, k] += 1.0
    assert bench.sampled_rel_err(Ct, o) > 1e-6


def test_oracle_sample_takes_given_inputs_and_reports_each_result():
    import numpy as np

    from oracle import tproduct as O
    specs = synth.batched_specs(512, 0)[:3]
    given = {}

    def inputs(i):
        s = specs[i]
        given[i] = synth.normal(np.random.Generator(np.random.PCG64(i)), (s.n1, s.n2, s.n3))
        return given[i]

    seen = {}
    rate, sl, nt, secs = bench.oracle_sample(specs, 0, 0.0, max_items=2, inputs=inputs,
                                             check=lambda i, W: seen.setdefault(i, W))
    assert nt == 1 and sorted(seen) == [0] and rate > 0 and secs > 0
    assert sl == specs[0].n3 // 2 + 1
    np.testing.assert_allclose(seen[0], O.prox_tnn(given[0], specs[0].tau), rtol=0, atol=1e-12)


def test_peaks_come_from_the_measured_file_or_the_recorded_values(tmp_path):
    import json
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}))
    got = bench.load_peaks(str(p))
    assert (got["hbm_gbs"], got["bf16_tflops"], got["sm_max_mhz"]) == (7000.0, 2000.0, 2000.0)
    assert got["source"] == "MEASURED_PEAKS.json"
    miss = bench.load_peaks(str(tmp_path / "absent.json"))
    assert miss["source"].startswith("recorded") and miss["hbm_gbs"] == 6685.5
    # FP32 ALU peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
    assert abs(152 * 128 * 2 * 2.070e9 / 1e12 - 80.54784) < 1e-9


def test_learned_launch_count_ignores_split_launches():
    # the learned method's fallback groups are planned without splitting by CTA size, so the
    # bench counts them under the chosen shape with split_launches = 0 (measured: 240
    # launches over 10 steps under an autotuned shape that splits the plain path's launches)
    shapes = _batch_shapes()
    n3s = [s.n3 for s in synth.batched_specs(512, 0)]
    tuned = {"target_lane_pairs": 7, "max_warps": 32, "split_launches": 1}
    learned = dict(tuned, split_launches=0)
    assert bench.svd_launch_groups(shapes, tuned) >= bench.svd_launch_groups(shapes, learned)
    per_call = bench.LEARNED_FIXED_LAUNCHES + 2 * bench.dft_launches(n3s) + \
        bench.svd_launch_groups(shapes, learned)
    assert per_call * 10 == 240


def test_bench_options_parse():
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
        assert a.host_parts == 1 and a.stream_calls == 500
        assert tuple(int(v) for v in a.gemm_shape.split(",")) == (2048, 1024, 1024, 64)
        sys.argv = ["bench.py", "--host-parts", "2", "--gemm-shape", "1024,1024,512,32"]
        a = bench.parse()
        assert a.host_parts == 2 and a.gemm_shape == "1024,1024,512,32"
    finally:
        sys.argv = old
