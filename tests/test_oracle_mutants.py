"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them.

Each mutant is a copy of oracle.c with one textual change, compiled into a
temporary directory and exercised in a child process (a broken index could
read out of bounds), which reports how many pins failed.
"""
import json
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, replacement, occurrence index or None for all)
MUTANTS = [
    ("fft_twiddle_sign", "double ang = sign * 2.0 * PI * t / len;",
     "double ang = -sign * 2.0 * PI * t / len;", None),
    ("fft_butterfly_sign", "x[2 * b] = x[2 * a] - br;", "x[2 * b] = x[2 * a] + br;", None),
    ("range_window_dropped", "out[2 * n] = w_r[n] * in[2 * n];",
     "out[2 * n] = in[2 * n];", None),
    ("lerp_weights_swapped", "*vr = (1.0 - f) * s[2 * i0] + f * s[2 * i0 + 2];",
     "*vr = f * s[2 * i0] + (1.0 - f) * s[2 * i0 + 2];", None),
    ("lerp_wrong_neighbour", "*vi = (1.0 - f) * s[2 * i0 + 1] + f * s[2 * i0 + 3];",
     "*vi = (1.0 - f) * s[2 * i0 + 1] + f * s[2 * i0 + 1];", None),
    ("bp_phase_sign", "const double a2 = sign * 2.0 * PI * f0 / c;",
     "const double a2 = -sign * 2.0 * PI * f0 / c;", None),
    ("bp_rx_uses_tx", "const double d_rx = hypot(x - qr[0], y - qr[1]);\n"
     "                const double d_hyp",
     "const double d_rx = hypot(x - q_tx[2 * m], y - q_tx[2 * m + 1]);\n"
     "                const double d_hyp", None),
    ("bp_a1_factor", "const double a1 = slope * n_fft / (c * fs);",
     "const double a1 = slope * n_fft / (2.0 * c * fs);", None),
    ("bp_window_dropped", "const double w = w_az ? w_az[m] : 1.0;\n"
     "            for (int n = 0; n < R; ++n) {\n"
     "                const double *qr = q_rx + 2 * ((long long)m * R + n);\n"
     "                const double d_rx",
     "const double w = 1.0;\n"
     "            for (int n = 0; n < R; ++n) {\n"
     "                const double *qr = q_rx + 2 * ((long long)m * R + n);\n"
     "                const double d_rx", 0),
    ("crop_upper_inclusive", "if (!(fl >= crop_lo && fl < crop_hi)) return 0;",
     "if (!(fl >= crop_lo && fl <= crop_hi)) return 0;", None),
    ("alg1_f0_dropped", "const double ph = sign * 2.0 * PI * f0 * tau;",
     "const double ph = sign * 2.0 * PI * tau;", None),
    ("alg1_doppler_sign", "const double f_hyp = slope * tau + f0 * (v_tx + v_rx) / c;",
     "const double f_hyp = slope * tau - f0 * (v_tx + v_rx) / c;", None),
    ("alg1_rx_velocity_dropped", "const double f_hyp = slope * tau + f0 * (v_tx + v_rx) / c;",
     "const double f_hyp = slope * tau + f0 * v_tx / c;", None),
    ("time_origin_rotation_sign", "const double ang = -sign * 2.0 * PI * t0 * k / nfft;",
     "const double ang = sign * 2.0 * PI * t0 * k / nfft;", None),
    ("mf_frequency_scale", "const double cyc = slope * d / (c * fs);",
     "const double cyc = slope * d / (c * fs) * 1.01;", None),
    ("mf_phase_sign", "ph *= sign * 2.0 * PI;", "ph *= -sign * 2.0 * PI;", None),
    ("hann_period", "w[n] = 0.5 - 0.5 * cos(2.0 * PI * n / (L - 1));",
     "w[n] = 0.5 - 0.5 * cos(2.0 * PI * n / L);", None),
    ("sum_over_rx_truncated", "for (int n = 0; n < R; ++n) {\n"
     "                const double *qr = q_rx + 2 * ((long long)m * R + n);\n"
     "                const double d_rx = hypot(x - qr[0], y - qr[1]);\n"
     "                const double d_hyp",
     "for (int n = 0; n < R - 1; ++n) {\n"
     "                const double *qr = q_rx + 2 * ((long long)m * R + n);\n"
     "                const double d_rx = hypot(x - qr[0], y - qr[1]);\n"
     "                const double d_hyp", None),
    ("polar_range_resolution_halved", "const double dr = c / (2.0 * B) / factor;",
     "const double dr = c / B / factor;", None),
    ("polar_wavelength_at_f0", "const double fc = f0 + slope * N / (2.0 * fs);",
     "const double fc = f0;", None),
    ("polar_azimuth_resolution_full_aperture", "const double dphi = (c / fc) / (2.0 * L) / factor;",
     "const double dphi = (c / fc) / L / factor;", None),
    ("polar_origin_first_chirp", "const double ox = 0.5 * (q_tx[0] + q_tx[2 * (M - 1)]);",
     "const double ox = q_tx[0];", None),
    ("polar_half_circle", "jhi = (long long)ceil(PI / dphi) - 1;", "jhi = 0;", None),
    ("doppler_sign", "out[p] = f0 * (-(v_tx + v_rx)) / c * n_fft / fs;",
     "out[p] = f0 * (v_tx + v_rx) / c * n_fft / fs;", None),
    ("doppler_rx_term_dropped", "out[p] = f0 * (-(v_tx + v_rx)) / c * n_fft / fs;",
     "out[p] = f0 * (-(2.0 * v_tx)) / c * n_fft / fs;", None),
    ("doppler_rx_mean_per_chirp_only", "rx /= (double)M * R; ry /= (double)M * R;",
     "rx /= M; ry /= M;", None),
    ("doppler_bins_scale", "out[p] = f0 * (-(v_tx + v_rx)) / c * n_fft / fs;",
     "out[p] = f0 * (-(v_tx + v_rx)) / c / fs;", None),
]

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import oracle
from tests.oracle_pins import ALL_PINS
lib = oracle.load({path!r})
failed = []
for pin in ALL_PINS:
    try:
        pin(lib)
    except Exception as e:
        failed.append(pin.__name__)
print(json.dumps(failed))
"""


def _mutate(text, old, new, occurrence):
    assert old in text, f"mutation anchor not found: {old[:60]!r}"
    if occurrence is None:
        return text.replace(old, new)
    parts = text.split(old)
    return old.join(parts[:occurrence + 1]) + new + old.join(parts[occurrence + 1:])


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, occ):
    text = open(SRC).read()
    mutated = _mutate(text, old, new, occ)
    assert mutated != text
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "oracle_mut.c")
        with open(src, "w") as f:
            f.write(mutated)
        lib = oracle.build(force=True, src=src, out=os.path.join(td, "libmut.so"))
        proc = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, path=lib)],
                              capture_output=True, text=True, timeout=300)
    if proc.returncode != 0:
        # a crash of the mutant counts as caught
        return
    failed = json.loads(proc.stdout.strip().splitlines()[-1])
    assert failed, f"mutant {name} passed every pin"


def test_unmutated_passes_in_child():
    proc = subprocess.run([sys.executable, "-c",
                           CHILD.format(root=ROOT, path=oracle.build())],
                          capture_output=True, text=True, timeout=300)
    assert proc.returncode == 0, proc.stderr
    assert json.loads(proc.stdout.strip().splitlines()[-1]) == []
