"""Shared test utilities: device copies of synthetic inputs and dense views
of collected results.  Imports the product binding and the oracle side by
side; neither imports the other."""

import numpy as np
import torch

from oracle.graph import csc_to_dense


def to_device(csr, dev="cuda"):
    import paper_2212_01997_gb300 as gb
    return gb.DeviceCSR.from_arrays(csr.n, csr.indptr, csr.indices, csr.data, dev)


def dense_result(csc, val=None):
    v = (csc.val if val is None else val).cpu().numpy()
    return csc_to_dense(csc.n, csc.ptr.cpu().numpy(), csc.idx.cpu().numpy(), v)


def max_abs_block_error(R, ref, part):
    """max |GPU - oracle| over D and every D1 (collected, element by element)."""
    n = part.n
    D = dense_result(R.D)
    eD = np.abs(D - csc_to_dense(n, *ref.D)).max()
    eD1 = max([np.abs(dense_result(R.D, d.val) - csc_to_dense(n, *r)).max()
               for d, r in zip(R.D1, ref.D1)] + [0.0])
    return eD, eD1
