"""GB300-native batched adaptive cubature of Brillouin-zone bubble integrals
(the PAID hot path).  The CUDA library is loaded on first use by
``paper_1610_09991_gb300.paid``; ``workloads`` builds seeded inputs."""
