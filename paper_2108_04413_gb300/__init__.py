"""GB300-native Pauli-exponential state-vector engine after QForte (arXiv:2108.04413).

* `qf`      -- ctypes binding of libqf (the C ABI in include/qf.h); importing it
               raises if the CUDA library has not been built.
* `prep`    -- host-side problem preparation: Jordan-Wigner images of the
               molecular Hamiltonian and of dUCC excitations, random circuits.
* `autograd`-- torch.autograd.Function over qf_energy_grad.
* `serving` -- continuous-batching energy+gradient server.
"""
