"""GB300-native exact projection of piecewise-linear simplicial meshes onto regular grids."""
