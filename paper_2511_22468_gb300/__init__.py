"""GB300-native differentiable direct-sum N-body (arXiv 2511.22468, "Odisseo").

The compute path is the C-ABI library ``libnbody.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``nbody`` is its thin Python binding.  Importing
this package does not load the library; the first call into ``nbody`` does,
and raises if the library is missing.
"""
