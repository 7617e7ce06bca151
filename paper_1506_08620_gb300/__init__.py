"""Direct search (Cannizzo, arXiv 1506.08620) as a GB300-native CUDA library."""
