"""Compile and run the ALU / copy peak microbenchmark (tools/alu_peaks.cu) on the current GPU.

    python -m paper_2305_08986_gb300.tools.peaks
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    src = os.path.join(HERE, "alu_peaks.cu")
    exe = os.path.join(tempfile.mkdtemp(), "alu_peaks")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    sys.exit(r.returncode)


if __name__ == "__main__":
    main()
