"""bench.py's bookkeeping on the CPU: the algorithmic byte counts of the fused
step (Sec. 3.2, Eq. traffic with kappa = 5), the stored ncu traffic record
(it must belong to the committed step sources and to the workload's shape),
and the time-to-solution forms the default line runs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

D, NNZ, NB = 128 ** 3, 7 * 128 ** 3, 64


def test_generic_step_bytes_of_the_stencil():
    # nnz (S_v + 4) + 5 nb D S_x: 14,680,064 * 8 + 5 * 64 * 2,097,152 * 4 (FP32)
    assert bench.generic_step_bytes(D, NNZ, NB, 4.0) == 117_440_512 + 2_684_354_560
    assert bench.generic_step_bytes(D, NNZ, NB, 8.0) == 14_680_064 * 12 + 5 * 64 * 2_097_152 * 8


def test_filter_bytes_sums_the_steps():
    # step 1 reads x_0 and writes x_1; step 2 reads x_1, x_0 and writes x_2 and
    # the accumulator; generic steps move five vectors, the last four
    for n in (2, 3, 4, 500):
        mat = NNZ * 8.0
        vec = NB * D * 4.0
        want = (mat + 2 * vec) + (mat + (4 if n > 2 else 3) * vec)
        want += max(0, n - 3) * (mat + 5 * vec) + (mat + 4 * vec if n >= 3 else 0)
        assert bench.filter_bytes(D, NNZ, NB, n, 4.0) == want


def test_traffic_record_belongs_to_the_committed_kernel():
    """roofline.traffic is an ncu capture of one generic FP32 step on this
    shape; it is only valid for the step sources it was taken on."""
    t = bench.TRAFFIC_F32
    assert (t["rows"], t["nnz"], t["nb"]) == (D, NNZ, NB)
    assert t["sources_sha256"] == bench.step_sources_sha256()
    got, why = bench.traffic_record(D, NNZ, NB)
    assert got == t["bytes"] and "ncu" in why
    # within a few percent of the algorithmic bytes (no wasted re-reads)
    alg = bench.generic_step_bytes(D, NNZ, NB, 4.0)
    assert 0.95 * alg <= got <= 1.05 * alg
    assert bench.traffic_record(D, NNZ, 32)[0] is None


def test_default_time_to_solution_forms_exist():
    src = open(os.path.join(ROOT, "bench.py")).read()
    key = '"--tts-forms-bench", default="'
    i = src.index(key) + len(key)
    forms = src[i:src.index('"', i)].split(",")
    assert forms and all(f in bench.TTS_FORMS for f in forms)
    # each form: (precision, learned constants, intervals, finish)
    for prec, learned, iv, finish in bench.TTS_FORMS.values():
        assert prec in ("f64", "f32", "ff") and iv in ("ritz", "lehmann") and finish in ("f64", "ff")
