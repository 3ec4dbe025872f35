"""GB300-native PanDelos-plus hot path: exact generalized Jaccard of k-mer
multiplicity profiles between genome pairs, Best Hits and Bidirectional Best
Hits, computed by hand-written CUDA kernels (sm_103a) behind a C ABI."""
