"""Stored oracle values for the GPU parity tests (written by
tests/golden/make_oracle_samples.py from the CPU oracle alone), and the error
measures of Section 4."""
import importlib.util
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "make_oracle_samples", os.path.join(_HERE, "golden", "make_oracle_samples.py"))
samples = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(samples)

reference = samples.reference


def err2(got, ref):
    """Err_2 of Section 4: relative L2 error over the targets (vector 2-norms)."""
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def errmax(got, ref):
    """Err_max of Section 4: largest pointwise relative error over the targets."""
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return float(np.max(num / den))


def tables(name):
    z = np.load(os.path.join(_HERE, "golden", "oracle_%s.npz" % name))
    return {k: z[k] for k in z.files}
