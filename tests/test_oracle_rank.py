"""Pins of the oracle's biased-initial-condition ranking (Sec. III-C/D).

* the std-critic MLP equals the same network in torch float64 (an
  independent implementation of the layers);
* the softplus output is positive and equals log(1 + e^z) (closed form);
* the selection is the N largest scores, ties taken by the lower index
  (checked by brute force on a small set with planted ties).
"""
import numpy as np
import pytest

import oracle
from paper_2602_19699_gb300 import workload as W


def test_std_critic_matches_torch():
    torch = pytest.importorskip("torch")
    n_in = 6
    w = W.std_critic_weights(n_in, seed=3).astype(np.float64)
    X = np.random.default_rng(0).normal(size=(50, n_in))
    o = 0
    net = torch.nn.Sequential(torch.nn.Linear(n_in, 256), torch.nn.Tanh(), torch.nn.Linear(256, 256), torch.nn.Tanh(),
                              torch.nn.Linear(256, 1), torch.nn.Softplus()).double()
    with torch.no_grad():
        for lin, (fi, fo) in zip([net[0], net[2], net[4]], [(n_in, 256), (256, 256), (256, 1)]):
            lin.weight.copy_(torch.from_numpy(w[o:o + fo * fi].reshape(fo, fi))); o += fo * fi
            lin.bias.copy_(torch.from_numpy(w[o:o + fo])); o += fo
        ref = net(torch.from_numpy(X)).numpy()[:, 0]
    np.testing.assert_allclose(oracle.std_critic(w, X), ref, rtol=1e-12)


def test_selection_brute_force_with_ties():
    n_in = 3
    w = W.std_critic_weights(n_in, seed=4)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(40, n_in))
    X[7] = X[3]; X[20] = X[3]; X[31] = X[11]          # identical candidates -> tied scores
    s = oracle.std_critic(w, X)
    assert np.all(s > 0)
    for N in (1, 3, 4, 10, 40):
        idx, _ = oracle.rank_candidates(w, X, N)
        # brute force: candidate i is chosen iff fewer than N candidates beat it,
        # where j beats i when s_j > s_i or (s_j == s_i and j < i)
        beats = np.array([np.sum((s > s[i]) | ((s == s[i]) & (np.arange(40) < i))) for i in range(40)])
        np.testing.assert_array_equal(idx, np.where(beats < N)[0])
