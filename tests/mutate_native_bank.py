"""Mutation check of the native bank structuring (run by hand: python tests/mutate_native_bank.py).

`rf_bank_structure` is host code, so its CPU tests (tests/test_bank.py, against the oracle and
hand-worked banks) can be checked the same way as the oracle's pins.  This script plants one
plausible mistake at a time in a scratch copy of csrc/bank.cu, compiles that file alone and relinks
it with the objects of an existing in-tree build, then runs tests/test_bank.py against the result.
The exit status is non-zero if a mistake survives.  Needs nvcc and a built library.
"""
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2511_12894_gb300")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (text in bank.cu, planted replacement, what the mistake is)
M = [
 ("const size_t h = idx.size() / 2;", "const size_t h = (idx.size() + 1) / 2;", "split extra in first half"),
 ("if (best < 0 || s < best_sum - 1e-9 * best_sum) {", "if (best < 0 || s > best_sum + 1e-9 * best_sum) {", "reference maximises"),
 ("} else if (std::fabs(s - best_sum) <= 1e-9 * best_sum && i < best) {", "} else if (std::fabs(s - best_sum) <= 1e-9 * best_sum && i > best) {", "tie to highest index"),
 ("mc[i] = std::pow(m1 * m2, 0.6) / std::pow(m1 + m2, 0.2);", "mc[i] = std::pow(m1 * m2, 0.6) / std::pow(m1 + m2, 0.4);", "chirp mass exponent"),
 ("eta[i] = m1 * m2 / ((m1 + m2) * (m1 + m2));", "eta[i] = m1 * m2 / (m1 + m2);", "eta definition"),
 ("return hi - lo <= max_spread;", "return hi - lo < max_spread;", "spread limit strict"),
 ("return (int64_t)x.size() <= max_size;", "return (int64_t)x.size() < max_size;", "size limit strict"),
 ("tau[i] = -(tf2_dphase(make_tf2(t, pn_order), f_low) / kTwoPi);", "tau[i] = (tf2_dphase(make_tf2(t, pn_order), f_low) / kTwoPi);", "duration sign"),
 ("    t.tc = 0.0;\n", "", "duration with the template's tc"),
 ("return mc[a] < mc[b] || (mc[a] == mc[b] && a < b);", "return mc[a] < mc[b] || (mc[a] == mc[b] && a > b);", "chirp-mass tie order"),
 ("return eta[a] < eta[b] || (eta[a] == eta[b] && a < b);", "return eta[a] > eta[b] || (eta[a] == eta[b] && a < b);", "eta order reversed"),
]


def main() -> int:
    sys.path.insert(0, ROOT)
    from paper_2511_12894_gb300 import build
    build.build()
    nvcc = build.nvcc()
    scratch = tempfile.mkdtemp(prefix="bank_mutants_")
    try:
        for d in ("oracle", "workload", "tests", "include"):
            shutil.copytree(os.path.join(ROOT, d), os.path.join(scratch, d), ignore=shutil.ignore_patterns("__pycache__"))
        pkg = os.path.join(scratch, "paper_2511_12894_gb300")
        shutil.copytree(PKG, pkg, ignore=shutil.ignore_patterns("__pycache__"))
        src = os.path.join(pkg, "csrc", "bank.cu")
        orig = open(src).read()
        objdir = os.path.join(pkg, "_build")
        objs = [os.path.join(objdir, f) for f in sorted(os.listdir(objdir)) if f.endswith(".o") and f != "bank.o"]
        flags = [*ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                 "-I", os.path.join(scratch, "include"), "-I", os.path.join(pkg, "csrc")]
        lib = os.path.join(pkg, "librf.so")
        env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
        survivors = []
        for old, new, name in M:
            if orig.count(old) != 1:
                print(f"{'absent':9s} {name}")
                survivors.append(name)
                continue
            open(src, "w").write(orig.replace(old, new, 1))
            t0 = time.time()
            obj = os.path.join(scratch, "bank_mutant.o")
            subprocess.run([nvcc, *flags, "-c", src, "-o", obj], check=True, capture_output=True)
            subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", lib, *objs, obj], check=True,
                           capture_output=True)
            os.utime(lib, None)   # newer than every source, so the tests' build() keeps it
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                                "tests/test_bank.py"], cwd=scratch, capture_output=True, text=True, timeout=600,
                               env=env)
            caught = r.returncode != 0
            if not caught:
                survivors.append(name)
            by = next((ln.split(" - ")[0] for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))), "")
            print(f"{'caught' if caught else 'SURVIVED':9s} {name:36s} {time.time() - t0:5.1f}s {by}", flush=True)
        print(f"{len(M)} planted mistakes, {len(survivors)} not caught")
        return 1 if survivors else 0
    finally:
        shutil.rmtree(scratch, ignore_errors=True)


if __name__ == "__main__":
    sys.exit(main())
