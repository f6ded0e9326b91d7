"""GB300-native exact ddKS (arXiv 2106.13706).  The binding is added with the CUDA library."""
