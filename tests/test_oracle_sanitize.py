"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU only).

tests/oracle_sanitize_driver.c calls every oracle function on seeded small graphs (all
option settings, empty inputs, self-loops, duplicates, unlabelled nodes, empty classes,
invalid inputs); any out-of-bounds access, leak, undefined operation or failed check ends
it with a non-zero status.  Skipped where gcc cannot build with the sanitizers."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / "oracle_sanitize")
    cmd = [gcc, "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-ffp-contract=off",
           os.path.join(ROOT, "oracle", "gee_oracle.c"), os.path.join(ROOT, "oracle", "gee_oracle_rows.c"),
           os.path.join(HERE, "oracle_sanitize_driver.c"), "-o", exe, "-pthread", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"no sanitizer build here: {r.stderr.strip()[:200]}")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "all checks passed" in run.stdout
