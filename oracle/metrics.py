"""Quality metrics of §4 (arXiv 2103.11847), float64 (oracle).

Test infrastructure only: see the package docstring.

  Relative error = ||X_hat - X_restored||_F / ||X_hat||_F.
  SNR(X_restored) = 10 log10(||X_hat - E(X_hat)||_F^2 / ||X_restored - X_hat||_F^2),
  E(X_hat) the mean grey level of the clean image; the paper does not say over
  which entries, so it is the mean over all entries of all channels.
"""
import numpy as np


def relative_error(X_true, X):
    X_true = np.asarray(X_true, np.float64)
    return float(np.linalg.norm((X_true - np.asarray(X, np.float64)).ravel())
                 / np.linalg.norm(X_true.ravel()))


def snr_db(X_true, X):
    X_true = np.asarray(X_true, np.float64)
    num = np.sum((X_true - X_true.mean()) ** 2)
    den = np.sum((np.asarray(X, np.float64) - X_true) ** 2)
    return float(10.0 * np.log10(num / den))
